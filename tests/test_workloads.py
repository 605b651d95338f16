"""The synthetic workloads are fixed: the bench line, the parity tests and the
committed selector data all refer to exactly these matrices and vectors.  A
change of the generators must be deliberate, so their output is pinned by
size and a SHA-1 of the arrays (row_ptr int32, col int32, val float64 bytes),
generated here without the on-disk cache.  The fingerprints were recorded
from synth/ when the current measurements were taken."""
import gzip
import hashlib
import json
import os

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def fingerprint(A) -> str:
    h = hashlib.sha1()
    for a in (A.row_ptr.astype(np.int32), A.col.astype(np.int32), A.val.astype(np.float64)):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


@pytest.mark.parametrize("name, make, n, nnz, fp", [
    ("stencil7_32", lambda: synth.stencil_3d(32, 32, 32, 7, seed=0),
     32768, 223232, "996a0ebb98822c5f"),
    ("stencil27_128", lambda: synth.stencil_3d(128, 128, 128, 27, seed=1, drop_rate=0.3,
                                               drop_block=4096, offband_row_frac=0.01,
                                               offband_per_row=2),
     2097152, 39894869, "4395161c16d80dd7"),
    ("scattered_4m", lambda: synth.scattered_diagonals(4194304, 19, 20000, 0.6, 2048, 3.0,
                                                       seed=2),
     4194304, 60899659, "c984cd896f09c68e"),
])
def test_named_workloads_are_fixed(name, make, n, nnz, fp):
    A = make()
    assert (A.n, A.nnz) == (n, nnz), name
    assert fingerprint(A) == fp, name
    # config_matrix builds the same recipe (possibly from its cache)
    B = synth.config_matrix(name)
    assert (B.n, B.nnz) == (n, nnz) and fingerprint(B) == fp, name


def test_vectors_are_fixed():
    assert hashlib.sha1(synth.uniform_vector(4096, 1).tobytes()).hexdigest()[:16] == "70c616fd8c6b9fe0"
    assert hashlib.sha1(synth.loguniform_vector(4096, 2).tobytes()).hexdigest()[:16] == "68fed74f94583a87"


@pytest.mark.parametrize("split, base", [("train", 1000), ("test", 9000)])
def test_selector_data_came_from_this_family(split, base):
    # the committed timing records name their family member; the generator
    # must still produce the matrix of that size
    path = os.path.join(ROOT, "paper_2105_04937_gb300", "selector_data", f"{split}.jsonl.gz")
    with gzip.open(path, "rt") as f:
        recs = [json.loads(next(f)) for _ in range(4)]
    for r in recs:
        p = synth.family_params(r["idx"], base_seed=base)
        assert p == r["params"], (split, r["idx"])
        A = synth.family_matrix(p)
        assert (A.n, A.nnz) == (r["n"], r["nnz"]), (split, r["idx"])
    A0 = synth.family_matrix(synth.family_params(0, base_seed=base))
    assert fingerprint(A0) == {"train": "8d38e6f2639836e5", "test": "0da2aeb786120b59"}[split]
