"""CPU replay of the staged-x kernel's index arithmetic and ring protocol
(k_mhdc_spmv_xw, variants 16-19), written out from the kernel's rules:

* windows: a unit of R rows at x index a0 reads x[a0 + off_p, a0 + off_p + R)
  for each diagonal p of its block; a window starts at (a0 + off) rounded
  down to V elements (16 bytes) and takes diagonals while (a0 + off_p + R)
  rounded up to V stays within base + XCAP - V; each window copies its
  in-range part [max(base, 0), min(end, n rounded down to V)).
* rings: the producer issues x windows up to XSTAGES - 2 windows ahead of the
  window whose values it issues; consumers wait for a window's first value
  stage, then release the previous window, then wait for the window.

Checked here: every copy in bounds, 16-byte aligned and inside its slot;
every shared-memory read (a misaligned vector reads the two aligned 16-byte
vectors around it) inside its slot and, for the elements used, inside the
copied range; and the two rings never deadlock at that look-ahead -- while
one window more does deadlock (so the simulation can see a deadlock).
Windows whose end is rounded up to 16 bytes already cover the second vector
of a misaligned read, so the XCAP - V limit keeps one vector to spare.  The
GPU tests check the kernel's results; this checks the reasoning that made its
first run safe (copying up to n instead of n rounded down to 16 bytes, for
one, fails it)."""
import numpy as np
import pytest

import oracle
import synth

CONFIGS = [(4, 2, 8, 4), (8, 1, 8, 4), (4, 1, 12, 6), (8, 2, 6, 3)]  # (NCW, U, DSTAGES, XSTAGES)


def unit_windows(M, V, R, XW):
    """Per unit: (a0, rows in unit, [(first diagonal, end, base)...])."""
    n, n_b = M["n"], M["bl"]
    dptr = np.asarray(M["dia_ptr"], np.int64)
    doff = np.asarray(M["dia_offset"], np.int64)
    upb = -(-n_b // R)
    out = []
    for u in range(upb * (-(-n // n_b))):
        ib, t0 = divmod(u, upb)
        t0 *= R
        r0 = ib * n_b
        rows = min(n - r0, n_b)
        if t0 >= rows:
            continue
        a0 = r0 + t0
        p, p1 = int(dptr[ib]), int(dptr[ib + 1])
        wins = []
        while p < p1:
            base = (a0 + int(doff[p])) & -V
            q = p + 1
            while q < p1 and ((a0 + int(doff[q]) + R + V - 1) & -V) - base <= XW:
                q += 1
            wins.append((p, q, base))
            p = q
        out.append((a0, min(rows - t0, R), wins))
    return out


def check_arithmetic(M, esize, NCW, U):
    V = 16 // esize
    NT = NCW * 32
    R = NT * U * V
    XCAP = R + 512
    XW = XCAP - V
    n = M["n"]
    nV = n & -V
    doff = np.asarray(M["dia_offset"], np.int64)
    P = int(np.asarray(M["dia_ptr"])[-1])
    # first row (in the unit) of each lane's vectors, by vector k, warp, lane
    tl = (np.arange(NT * U) * V).reshape(U, NCW, 32)
    offs = np.arange(V)
    for a0, ru, wins in unit_windows(M, V, R, XW):
        nbytes = (ru * esize + 15) & ~15
        for p, q, base in wins:
            wend = (a0 + int(doff[q - 1]) + R + V - 1) & -V
            lo, hi = max(base, 0), min(wend, nV)
            if hi > lo:
                assert lo % V == 0 and hi % V == 0 and hi <= n
                assert 0 <= lo - base and hi - base <= XCAP
            for d in range(p, q):
                t0 = a0 - (a0 // M["bl"]) * M["bl"]
                start = (d * M["bl"] + t0) * esize
                assert start % 16 == 0 and start + nbytes <= P * M["bl"] * esize
                a = a0 + int(doff[d])
                e0 = a - base
                r = e0 % V
                jw = a + tl[:, :, 0]                               # per (vector, warp)
                fast = (jw >= 0) & (jw + 32 * V <= nV)
                used = a + tl[..., None] + offs                    # elements each lane uses
                if fast.any():
                    first = e0 + tl[fast] - (0 if (r == 0 or V == 2) else r)
                    last = first + (V if (r == 0 or V == 2) else 2 * V)
                    assert first.min() >= 0 and last.max() <= XCAP
                    uf = used[fast]
                    assert uf.min() >= lo and uf.max() < hi
                if not fast.all():
                    us = used[~fast]
                    sm = (us >= 0) & (us < nV)
                    assert np.all(us[sm] >= lo) and np.all(us[sm] < hi)


def rings_finish(win_sizes, DST, XST, XLOOK):
    """Discrete simulation of one CTA; False on a state where nobody moves."""
    W = len(win_sizes)
    diag_win = [w for w in range(W) for _ in range(win_sizes[w])]
    D = len(diag_win)
    x_iss = d_iss = x_rel = d_rel = c = dg = in_win = 0
    held = -1
    while c < D or x_iss < W or d_iss < D:
        moved = False
        while x_iss < W and x_iss <= dg + XLOOK and x_iss - XST < x_rel:
            x_iss += 1
            moved = True
        if dg < W and (x_iss == W or x_iss > dg + XLOOK) and d_iss - DST < d_rel:
            d_iss += 1
            in_win += 1
            moved = True
            if in_win == win_sizes[dg]:
                dg, in_win = dg + 1, 0
        if c < D:
            w = diag_win[c]
            if w != held and d_iss > c:
                if held >= 0 and x_rel == held:
                    x_rel += 1
                    moved = True
                if (held < 0 or x_rel > held) and x_iss > w:
                    held = w
            if held == w and d_iss > c:
                c += 1
                d_rel += 1
                moved = True
        elif held >= 0 and x_rel == held:
            x_rel += 1
            moved = True
        if not moved:
            return False
    return True


@pytest.fixture(scope="module")
def cases():
    rng = synth.Rng(5, 41)
    out = [(synth.config_matrix("stencil27_128", 0.25), 4096, 0.6),
           (synth.config_matrix("scattered_4m", 1 / 128), 2048, 0.6),
           (synth.paper_stencil(20001, 3), 4096, 0.0)]
    for seed in range(2):
        n = int(rng.integers(1, 1, 3000)[0])
        A = synth.random_sparse(n, 0.01, seed=300 + seed, diag_bias=0.7)
        out += [(A, 64, 0.0), (A, 1024, 0.5), (A, 3 * n + 8, 0.1)]
        B = synth.random_sparse(int(n // 8) + 1, 0.02, seed=400 + seed, diag_bias=0.7)
        out.append((B, 8, 0.0))     # 8-row blocks: one unit per block
    return out


def test_window_arithmetic_stays_in_bounds(cases):
    for A, n_b, theta in cases:
        for esize, dt in ((8, "f64"), (4, "f32"), (2, "bf16")):
            if (n_b * esize) % 16:
                continue
            M = oracle.convert(A, n_b, theta, dt)
            for NCW, U, _, _ in CONFIGS:
                check_arithmetic(M, esize, NCW, U)


def test_rings_never_deadlock_at_the_kernels_lookahead(cases):
    for A, n_b, theta in cases[:3]:
        M = oracle.convert(A, n_b, theta, "f64")
        for NCW, U, DST, XST in CONFIGS:
            R = NCW * 32 * U * 2
            units = unit_windows(M, 2, R, R + 512 - 2)
            for b, grid in ((0, 1), (1, 3), (7, 456)):
                sizes = [q - p for _, _, wins in units[b::grid] for p, q, _ in wins]
                assert rings_finish(sizes, DST, XST, XST - 2), (A.n, n_b, NCW, U, b, grid)
    # one window further ahead deadlocks on the stencil (the simulation can fail)
    M = oracle.convert(cases[0][0], 4096, 0.6, "f64")
    sizes = [q - p for _, _, wins in unit_windows(M, 2, 512, 1022) for p, q, _ in wins]
    assert not rings_finish(sizes, 8, 4, 3)
