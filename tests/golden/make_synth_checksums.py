"""Write ``synth_checksums.json``: a SHA-256 of every named workload's arrays.

    python tests/golden/make_synth_checksums.py

The generator feeds both the CUDA path and the oracle, so a change to it would
silently change every workload and every number measured on it; the test
``tests/test_synth.py::test_workload_checksums`` compares the generator's
current output with these stored digests.  This script calls only the
generator (no oracle, no CUDA library).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1308_4011_b300 import synth  # noqa: E402

FIELDS = ("method_class", "attr_class", "acc_rowptr", "acc_idx", "call_rowptr", "call_idx")


def system_digest(s) -> str:
    h = hashlib.sha256()
    h.update(np.asarray([s.n_classes, s.n_methods, s.n_attrs], dtype="<i8").tobytes())
    for f in FIELDS:
        a = getattr(s, f)
        h.update(np.asarray(a.shape, dtype="<i8").tobytes())
        h.update(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()


def arrays_digest(*arrs) -> str:
    h = hashlib.sha256()
    for a in arrs:
        h.update(np.asarray(a.shape, dtype="<i8").tobytes())
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def batched_digest(seeds) -> str:
    """One digest over the systems of a batched/served mix, in seed order."""
    h = hashlib.sha256()
    for seed in seeds:
        h.update(system_digest(synth.generate(**synth.batched_params(seed))).encode())
    return h.hexdigest()


def compute() -> dict:
    out = {}
    for name in ("tiny", "medium", "large"):
        out[name] = system_digest(synth.named(name))
    large = synth.named("large")
    rp, dst = synth.candidates(large, synth.LARGE_EXTRA_CANDIDATES, seed=synth.LARGE["seed"])
    out["large_candidates"] = arrays_digest(rp, dst)
    out["batched_seeds_100_355"] = batched_digest(range(100, 356))
    out["served_seeds_100_163"] = batched_digest(range(100, 164))
    return out


if __name__ == "__main__":
    path = os.path.join(HERE, "synth_checksums.json")
    with open(path, "w") as f:
        json.dump(compute(), f, indent=1, sort_keys=True)
        f.write("\n")
    print("wrote", path)
