"""The GPU-vs-oracle comparison rules themselves (tests/parity.py), on the CPU:
a correct result passes, and planted mistakes are reported, not excused."""
import numpy as np

import oracle
from tests import parity


def _c1(wl1):
    r = oracle.run_crsh(wl1.gbuffer, wl1.lights, wl1.shadow_cull, wl1.hash_lo, wl1.hash_hi, wl1.scene, wl1.bundle,
                        wl1.levels, wl1.build_pads())
    tri, t, u, v = r["hits"]
    return r, (tri.copy(), t.astype(np.float32), u.astype(np.float32), v.astype(np.float32))


def test_oracle_against_itself_passes(wl1):
    r, gpu = _c1(wl1)
    rep = parity.compare_hits(gpu, r["hits"], r["rays"], wl1.scene.verts)
    parity.check_report(rep)
    assert rep["ties"] == rep["edges"] == 0 and rep["hits"] > 50


def test_planted_wrong_triangle_is_unexplained(wl1):
    r, gpu = _c1(wl1)
    tri = gpu[0]
    hit = np.nonzero(tri >= 0)[0]
    i = hit[len(hit) // 2]
    tri[i] = (tri[i] + 1) % wl1.scene.n_tris        # a neighbour id the ray does not hit there
    miss = np.nonzero(r["hits"][0] < 0)[0]
    tri[miss[0]] = 5                                 # a hit where there is none
    rep = parity.compare_hits(gpu, r["hits"], r["rays"], wl1.scene.verts)
    bad = {u[0] for u in rep["unexplained"]}
    assert i in bad and miss[0] in bad


def test_planted_distance_error_is_caught(wl1):
    r, gpu = _c1(wl1)
    hit = np.nonzero(gpu[0] >= 0)[0]
    gpu[1][hit[0]] *= 1.0 + 3e-5
    gpu[2][hit[1]] += 3e-5
    rep = parity.compare_hits(gpu, r["hits"], r["rays"], wl1.scene.verts)
    assert rep["t_viol"] == 1 and rep["uv_viol"] == 1
