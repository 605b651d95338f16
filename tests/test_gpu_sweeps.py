"""The measurement modes of bench.py on tiny sizes: they run end to end and
their JSON lines hold the fields the summaries in profiles/ are made from."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stencil_sweep_small(tmp_path):
    out = tmp_path / "s.jsonl"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--sweep", "stencil",
                        "--sizes", "1e4,3e4", "--nb-n", "20000", "--out", str(out)],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    recs = [json.loads(l) for l in open(out)]
    st = [x for x in recs if x["sweep"] == "stencil"]
    assert len(st) == 6
    for x in st:
        assert x["dia_bits_equal_bdia"] and x["csr_within_tol"]
        assert set(x["gflops"]) == {"csr", "dia", "bdia", "mhdc"}
        assert 0 < x["model_paper_gamma"]["bdia_over_csr"] < 2
    nb = [x for x in recs if x["sweep"] == "stencil_nb"]
    assert len(nb) == 33 and all(x["max_abs_diff_vs_csr"] < 1e-9 for x in nb)
