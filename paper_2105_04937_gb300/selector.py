"""Learned parameter selector for M-HDC: data collection, training, evaluation.

The library measures the time of every candidate (n_b, theta, dtype) of its
grid on seeded matrices of a parametric family (mhdc_autotune), learns a small
MLP from the per-block diagonal-occupancy features (mhdc_features) to each
candidate's log time relative to the matrix's fastest (its own forward,
backward and Adam kernels, mhdc_mlp_*), and is scored by regret against the
exhaustive autotuner on held-out matrices, beside the paper's fixed policy
(theta = 0.6, one block width; Sec. 6.4.3) and the paper's byte model
(Sec. 5.3.3) used as a selector.

Records are JSON lines (one matrix per line), appended as they are measured,
so an interrupted collection resumes where it stopped.  Trained weights are
stored in a small versioned binary file with a SHA-256 checksum.
"""
from __future__ import annotations

import hashlib
import json
import os
import struct
import time

import numpy as np

from . import (MHDC_NUM_CANDIDATES, MHDC_NUM_FEATURES, MHDC_SELECT_MODEL, mhdc_autotune,
               mhdc_candidate, mhdc_features, mhdc_mlp_create, mhdc_mlp_forward,
               mhdc_mlp_get_params, mhdc_mlp_set_params, mhdc_mlp_train_step, mhdc_select)

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.bin")
MAGIC = b"MHDCMLP1"
TOLERANCES = {"fp64_only": 1e-12, "fp32_ok": 1e-5, "bf16_ok": 1e-1}
HIDDEN = 128


def _dtype_of(idx: int) -> str:
    return mhdc_candidate(idx)["dtype"]


def allowed_mask(tol: float, c: float) -> np.ndarray:
    """Candidates whose dtype's worst-case bound for rows of c terms is <= tol
    (the rule mhdc_select applies)."""
    ua = 2.0 ** -24
    k = c + 1
    g = k * ua / (1 - k * ua)
    bound = {"f64": 0.0, "f32": (1 + ua) ** 2 * (1 + g) - 1,
             "bf16": ((1 + ua) * (1 + 2.0 ** -8)) ** 2 * (1 + g) - 1}
    return np.array([bound[_dtype_of(i)] <= tol or _dtype_of(i) == "f64"
                     for i in range(MHDC_NUM_CANDIDATES)])


def paper_choice(tol: float, c: float) -> int:
    """Index of the paper's fixed policy: theta 0.6, n_b 4096, cheapest allowed dtype."""
    ok = allowed_mask(tol, c)
    for dt in ("bf16", "f32", "f64"):
        for i in range(MHDC_NUM_CANDIDATES):
            p = mhdc_candidate(i)
            if p["dtype"] == dt and p["n_b"] == 4096 and abs(p["theta"] - 0.6) < 1e-9 and ok[i]:
                return i
    raise RuntimeError("paper policy not in the candidate grid")


def _gen(idx_and_kw):
    """Worker: generate one family matrix on the CPU (runs in a spawned process)."""
    import synth
    idx, kw = idx_and_kw
    p = synth.family_params(idx, **kw)
    A = synth.family_matrix(p)
    return idx, p, A.n, A.row_ptr, A.col, A.val


def collect(indices, out_path, *, base_seed=1000, min_dim=32, max_dim=96, reps=10, workers=8,
            log=print, time_budget_s=None):
    """Measure features, candidate times and the model's choice for each family
    member in `indices`, appending JSON lines to out_path (skipping done ones)."""
    import multiprocessing as mp

    import torch
    done = set()
    if os.path.exists(out_path):
        with open(out_path) as f:
            for line in f:
                try:
                    done.add(json.loads(line)["idx"])
                except (ValueError, KeyError):
                    pass  # a partial last line from an interrupted run
    todo = [i for i in indices if i not in done]
    if not todo:
        return 0
    kw = dict(base_seed=base_seed, min_dim=min_dim, max_dim=max_dim)
    ctx = mp.get_context("spawn")
    t0 = time.time()
    n_done = 0
    with ctx.Pool(workers) as pool, open(out_path, "a") as out:
        for idx, p, n, rp, col, val in pool.imap(_gen, [(i, kw) for i in todo], chunksize=2):
            rpd = torch.from_numpy(rp).cuda()
            cold = torch.from_numpy(col).cuda()
            vald = torch.from_numpy(val).cuda()
            f = mhdc_features(n, rpd, cold)
            t = mhdc_autotune(n, rpd, cold, vald, reps=reps)
            nnz = int(rp[-1])
            model = {}
            for name, tol in TOLERANCES.items():
                sel = mhdc_select(n, rpd, cold, vald, tol, MHDC_SELECT_MODEL)
                model[name] = _index_of(sel)
            rec = dict(idx=idx, params=p, n=n, nnz=nnz, features=[float(v) for v in f],
                       times_us=[float(v) for v in t], model_choice=model)
            out.write(json.dumps(rec) + "\n")
            out.flush()
            n_done += 1
            if n_done % 50 == 0:
                log(f"collected {n_done}/{len(todo)} in {time.time() - t0:.0f}s")
            del rpd, cold, vald
            if time_budget_s and time.time() - t0 > time_budget_s:
                log(f"time budget reached after {n_done} matrices")
                break
    return n_done


def _index_of(sel: dict) -> int:
    for i in range(MHDC_NUM_CANDIDATES):
        p = mhdc_candidate(i)
        if p["dtype"] == sel["dtype"] and p["n_b"] == sel["n_b"] and abs(p["theta"] - sel["theta"]) < 1e-9:
            return i
    return -1


def load_records(path):
    import gzip
    recs = []
    opener = gzip.open if path.endswith(".gz") else open
    with opener(path, "rt") as f:
        for line in f:
            try:
                recs.append(json.loads(line))
            except ValueError:
                pass
    return recs


def dataset(recs):
    """Features X, targets T = log(t / t_min) and mask M (measured candidates)."""
    X = np.array([r["features"] for r in recs], dtype=np.float32)
    t = np.array([r["times_us"] for r in recs], dtype=np.float64)
    M = (t > 0).astype(np.float32)
    tmin = np.min(np.where(t > 0, t, np.inf), axis=1, keepdims=True)
    T = np.where(t > 0, np.log(np.maximum(t, 1e-9) / tmin), 0.0).astype(np.float32)
    return X, T, M, t


def train(recs, *, hidden=HIDDEN, epochs=400, batch=256, lr=1e-3, seed=7, log=print):
    """Train the selector network on the GPU with the library's own kernels."""
    import torch
    X, T, M, _ = dataset(recs)
    net = mhdc_mlp_create(MHDC_NUM_FEATURES, hidden, MHDC_NUM_CANDIDATES, seed=seed)
    Xd, Td, Md = (torch.from_numpy(a).cuda() for a in (X, T, M))
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            last = s + batch >= n
            loss = mhdc_mlp_train_step(net, Xd[idx].contiguous(), Td[idx].contiguous(),
                                       Md[idx].contiguous(), lr, want_loss=last)
        losses.append(loss)
        if log and (ep % 100 == 0 or ep == epochs - 1):
            log(f"epoch {ep}: loss {loss:.5f}")
    return net, losses


def predict(net, X):
    import torch
    return mhdc_mlp_forward(net, torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()).cpu().numpy()


def evaluate(net, recs):
    """Regret (t(choice) / t(best allowed) - 1) of the MLP, the paper's policy
    and the paper's model, per tolerance class, against the autotuner."""
    X, _, _, t = dataset(recs)
    pred = predict(net, X) if net is not None else None
    out = {}
    for name, tol in TOLERANCES.items():
        rg = {"mlp": [], "paper_policy": [], "paper_model": []}
        for r, (row_t, rec) in enumerate(zip(t, recs)):
            c = rec["nnz"] / rec["n"]
            ok = allowed_mask(tol, c) & (row_t > 0)
            best = np.min(row_t[ok])
            if pred is not None:
                pm = np.where(ok, pred[r], np.inf)
                rg["mlp"].append(row_t[int(np.argmin(pm))] / best - 1)
            pc = paper_choice(tol, c)
            rg["paper_policy"].append(row_t[pc] / best - 1 if row_t[pc] > 0 else np.nan)
            mc = rec["model_choice"][name]
            rg["paper_model"].append(row_t[mc] / best - 1 if mc >= 0 and row_t[mc] > 0 else np.nan)
        out[name] = {k: {"mean": float(np.nanmean(v)), "median": float(np.nanmedian(v)),
                         "p90": float(np.nanpercentile(v, 90)), "max": float(np.nanmax(v)),
                         "within_10pct": float(np.mean(np.array(v) <= 0.10))}
                     for k, v in rg.items() if v}
    return out


def save(net, path=WEIGHTS):
    p = mhdc_mlp_get_params(net)
    head = MAGIC + struct.pack("<iii", net.n_in, net.n_hidden, net.n_out)
    body = head + p.astype("<f4").tobytes()
    with open(path, "wb") as f:
        f.write(body + hashlib.sha256(body).digest())


def load(path=WEIGHTS):
    data = open(path, "rb").read()
    body, digest = data[:-32], data[-32:]
    if data[:8] != MAGIC or hashlib.sha256(body).digest() != digest:
        raise ValueError(f"{path}: not a selector weight file or corrupted")
    F, H, O = struct.unpack("<iii", body[8:20])
    net = mhdc_mlp_create(F, H, O)
    mhdc_mlp_set_params(net, np.frombuffer(body[20:], dtype="<f4"))
    return net
