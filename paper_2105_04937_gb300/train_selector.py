"""Command line for the learned selector: collect timings, train, evaluate.

  python -m paper_2105_04937_gb300.train_selector collect --data DIR --n-train 2000 --n-test 200
  python -m paper_2105_04937_gb300.train_selector train --data DIR [--weights FILE]
  python -m paper_2105_04937_gb300.train_selector evaluate --data DIR [--weights FILE]

Training matrices are family members 0..n_train-1 with seeds 1000 + idx,
held-out ones 0..n_test-1 with seeds 9000 + idx (see synth.family_params).
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["collect", "train", "evaluate", "all"])
    ap.add_argument("--data", required=True)
    ap.add_argument("--weights", default=None)
    ap.add_argument("--n-train", type=int, default=2000)
    ap.add_argument("--n-test", type=int, default=200)
    ap.add_argument("--min-dim", type=int, default=32)
    ap.add_argument("--max-dim", type=int, default=96)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 2))
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--time-budget", type=float, default=None, help="seconds for collection")
    a = ap.parse_args(argv)
    from paper_2105_04937_gb300 import selector as S
    os.makedirs(a.data, exist_ok=True)
    train_path = os.path.join(a.data, "train.jsonl")
    test_path = os.path.join(a.data, "test.jsonl")
    weights = a.weights or S.WEIGHTS
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    if a.cmd in ("collect", "all"):
        t0 = time.time()
        S.collect(range(a.n_test), test_path, base_seed=9000, min_dim=a.min_dim, max_dim=a.max_dim, reps=a.reps,
                  workers=a.workers, log=log, time_budget_s=a.time_budget)
        S.collect(range(a.n_train), train_path, base_seed=1000, min_dim=a.min_dim, max_dim=a.max_dim,
                  reps=a.reps, workers=a.workers, log=log,
                  time_budget_s=(a.time_budget - (time.time() - t0)) if a.time_budget else None)
        log(f"collection: {time.time() - t0:.0f}s")
    if a.cmd in ("train", "all"):
        recs = S.load_records(train_path)
        net, losses = S.train(recs, epochs=a.epochs, log=log)
        S.save(net, weights)
        log(f"trained on {len(recs)} matrices; final loss {losses[-1]:.5f}; saved {weights}")
    if a.cmd in ("evaluate", "all"):
        net = S.load(weights)
        tr = S.load_records(train_path)
        te = S.load_records(test_path)
        res = {"n_train": len(tr), "n_test": len(te), "held_out": S.evaluate(net, te),
               "train": S.evaluate(net, tr)}
        print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
