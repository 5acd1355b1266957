"""bench.py's host-side bookkeeping, on CPU: the launch count it claims per
pass, and when the committed DRAM-traffic record of the final-test kernel may
be attached to a bench line (only for the workload it was captured on, and
only while the kernel's source is the one the counters were taken from)."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_launches_per_pass():
    # hash_sort: tables, zeroing, gen, chunk, plan, 4 radix passes, chunk positions, gather = 11;
    # build: level 1 (with level 2) plus one per level above = L - 1;
    # traversal, word form: zeroing, mesh stage, top stage (5), 5 per level above 1, unit scan +
    # count + items at level 1; list form: 5 per level below the top plus the CSR pass;
    # closest hit: fill, final tests, finalize.
    assert bench.launches_per_step(4, True, True) == 11 + 3 + (2 + 5 + 5 * 2 + 3) + 3 == 37
    assert bench.launches_per_step(4, True, False) == 11 + 3 + (2 + 5 + 5 * 3 + 1) + 3 == 40
    assert bench.launches_per_step(4, False, True) == 36   # no chunk positions without compression
    assert bench.launches_per_step(1, True, True) == 11 + 1 + (2 + 5 + 1) + 3


def test_traffic_record_only_for_its_workload_and_source():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["k_closest_words"]
    src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    current = hashlib.sha256(src).hexdigest() == rec["source_sha256"]
    got = bench.closest_traffic("k_closest_words", rec["config"], None)
    assert got == (rec["bytes_per_launch"] if current else None)
    assert bench.closest_traffic("k_closest_words", rec["config"] + 1, None) is None   # another frame
    assert bench.closest_traffic("k_closest_words", rec["config"], 512) is None        # another resolution
    assert bench.closest_traffic("no_such_kernel", rec["config"], None) is None
