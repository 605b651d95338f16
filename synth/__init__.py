"""Seeded synthetic inputs for the M-HDC SpMV library and its oracle.

This module is shared by the oracle tests and by the CUDA path: it only makes
matrices and vectors, and holds none of the method's arithmetic (no diagonal
counting, selection, conversion or products).  Every random number comes from
SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based generator: output k of the
stream with key s is mix64(s + (k + 1) * 0x9E3779B97F4A7C15), so a draw depends
only on (seed, stream, index) and is the same on every machine.

Matrices are returned as :class:`CSR` with zero-based int32 ``row_ptr`` /
``col`` and float64 ``val``; columns are strictly increasing in every row and
no stored value is exactly zero.
"""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CSR", "Rng", "stencil_3d", "paper_stencil", "scattered_diagonals",
    "uniform_vector", "loguniform_vector", "config_matrix", "batch_matrices",
    "family_params", "family_matrix", "example_matrix", "dia_matrix", "paper_stencil_offsets",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


class Rng:
    """Counter-based SplitMix64 stream identified by (seed, stream)."""

    def __init__(self, seed: int, stream: int = 0):
        with np.errstate(over="ignore"):
            key = _mix64(np.array([(seed * 0x100000001B3 + stream) & ((1 << 64) - 1)],
                                  dtype=np.uint64))[0]
        self.key = np.uint64(key)
        self.ctr = 0

    def u64(self, k: int) -> np.ndarray:
        idx = np.arange(self.ctr + 1, self.ctr + 1 + k, dtype=np.uint64)
        self.ctr += k
        with np.errstate(over="ignore"):
            return _mix64(self.key + idx * _GOLDEN)

    def unit(self, k: int) -> np.ndarray:
        """Uniform doubles in [0, 1) with 53 random bits."""
        return (self.u64(k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform(self, k: int, lo: float, hi: float) -> np.ndarray:
        return lo + (hi - lo) * self.unit(k)

    def integers(self, k: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi) (multiply-high mapping of 32 random bits)."""
        span = np.uint64(hi - lo)
        r = self.u64(k) >> np.uint64(32)
        return (lo + ((r * span) >> np.uint64(32)).astype(np.int64)).astype(np.int64)

    def bernoulli(self, k: int, p: float) -> np.ndarray:
        return self.unit(k) < p

    def poisson(self, k: int, lam: float) -> np.ndarray:
        """Poisson(lam) by inversion of the cumulative distribution."""
        u = self.unit(k)
        kmax = int(lam + 12.0 * np.sqrt(lam + 1.0) + 12)
        pmf = np.empty(kmax + 1)
        pmf[0] = np.exp(-lam)
        for j in range(1, kmax + 1):
            pmf[j] = pmf[j - 1] * lam / j
        cdf = np.cumsum(pmf)
        cdf[-1] = 1.0
        return np.searchsorted(cdf, u, side="right").astype(np.int64)


@dataclass
class CSR:
    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col: np.ndarray      # int32[nnz]
    val: np.ndarray      # float64[nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def rows(self) -> np.ndarray:
        """Row index of every stored entry (int64)."""
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))


def _from_sorted_keys(n: int, keys: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    rows = keys // n
    col = (keys - rows * n).astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz does not fit in int32")
    return row_ptr.astype(np.int32), col


def _add_random_entries(n: int, keys: np.ndarray, rows_extra: np.ndarray,
                        rng: Rng) -> np.ndarray:
    """Add one uniform random column per entry of ``rows_extra`` (row ids,
    repeated for several entries per row) that collides neither with ``keys``
    (sorted, unique) nor with another added entry; collisions are redrawn."""
    if rows_extra.size == 0:
        return keys
    rows_extra = np.sort(rows_extra.astype(np.int64))
    cols = rng.integers(rows_extra.size, 0, n)
    new = rows_extra * n + cols
    while True:
        pos = np.searchsorted(keys, new)
        pos_c = np.minimum(pos, keys.size - 1)
        hit = keys[pos_c] == new
        order = np.argsort(new, kind="stable")
        srt = new[order]
        dup_sorted = np.zeros(new.size, dtype=bool)
        dup_sorted[1:] = srt[1:] == srt[:-1]
        dup = np.zeros(new.size, dtype=bool)
        dup[order] = dup_sorted
        bad = hit | dup
        nb = int(bad.sum())
        if nb == 0:
            break
        new[bad] = rows_extra[bad] * n + rng.integers(nb, 0, n)
    new.sort()
    merged = np.concatenate([keys, new])
    merged.sort(kind="stable")
    return merged


def _dominant_values(n: int, row_ptr: np.ndarray, col: np.ndarray, rng: Rng) -> np.ndarray:
    """Off-diagonal values U[-1, 1]; a_ii = 6 + |sum of the row's off-diagonals|."""
    nnz = int(row_ptr[-1])
    val = rng.uniform(nnz, -1.0, 1.0)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    is_diag = col.astype(np.int64) == rows
    off = np.where(is_diag, 0.0, val)
    rsum = np.bincount(rows, weights=off, minlength=n)
    val[is_diag] = 6.0 + np.abs(rsum[rows[is_diag]])
    # an exact zero would be dropped by the nonzero-set round trip: nudge it
    val[val == 0.0] = 2.0 ** -30
    return val


def _stencil_displacements(points: int) -> list[tuple[int, int, int]]:
    if points == 7:
        d = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    elif points == 13:
        d = [(0, 0, 0)]
        for s in (1, 2):
            d += [(s, 0, 0), (-s, 0, 0), (0, s, 0), (0, -s, 0), (0, 0, s), (0, 0, -s)]
    elif points == 27:
        d = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    else:
        raise ValueError("points must be 7, 13 or 27")
    # ascending column offset: order by (dz, dy, dx) since |dx| < nx, |dy| nx < nx ny
    return sorted(d, key=lambda t: (t[2], t[1], t[0]))


def stencil_3d(nx: int, ny: int, nz: int, points: int = 7, *, seed: int = 0,
               drop_rate: float = 0.0, drop_block: int = 4096,
               offband_row_frac: float = 0.0, offband_per_row: int = 0,
               offband_poisson: float = 0.0) -> CSR:
    """Finite-difference stencil on an nx*ny*nz grid with Dirichlet boundaries.

    Row i is grid point (x, y, z) with i = x + nx*(y + ny*z); a neighbour that
    falls outside the grid is dropped.  Optional partial-diagonal structure:
    each off-centre stencil offset is removed, with probability ``drop_rate``,
    from every ``drop_block``-row block independently.  Optional off-band
    entries: each row is picked with probability ``offband_row_frac`` and gets
    ``offband_per_row`` uniform random columns, and/or every row gets
    Poisson(``offband_poisson``) of them.  Values: off-diagonals U[-1, 1] and
    a_ii = 6 + |sum of the row's off-diagonals|.
    """
    n = nx * ny * nz
    rng_drop = Rng(seed, 1)
    rng_extra = Rng(seed, 2)
    rng_val = Rng(seed, 3)
    i = np.arange(n, dtype=np.int64)
    x = i % nx
    y = (i // nx) % ny
    z = i // (nx * ny)
    disp = _stencil_displacements(points)
    nblk = (n + drop_block - 1) // drop_block
    blk = i // drop_block
    cols = np.empty((n, len(disp)), dtype=np.int64)
    mask = np.empty((n, len(disp)), dtype=bool)
    for k, (dx, dy, dz) in enumerate(disp):
        ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny) & \
             (z + dz >= 0) & (z + dz < nz)
        if drop_rate > 0.0 and (dx, dy, dz) != (0, 0, 0):
            keep_blk = ~rng_drop.bernoulli(nblk, drop_rate)
            ok &= keep_blk[blk]
        cols[:, k] = i + dx + nx * (dy + ny * dz)
        mask[:, k] = ok
    keys = (i[:, None] * n + cols)[mask]  # row-major, ascending columns per row
    del cols, mask
    extra_rows = []
    if offband_row_frac > 0.0 and offband_per_row > 0:
        pick = np.nonzero(rng_extra.bernoulli(n, offband_row_frac))[0]
        extra_rows.append(np.repeat(pick, offband_per_row))
    if offband_poisson > 0.0:
        cnt = rng_extra.poisson(n, offband_poisson)
        extra_rows.append(np.repeat(i, cnt))
    if extra_rows:
        keys = _add_random_entries(n, keys, np.concatenate(extra_rows), rng_extra)
    row_ptr, col = _from_sorted_keys(n, keys)
    del keys
    val = _dominant_values(n, row_ptr, col, rng_val)
    return CSR(n, row_ptr, col, val,
               dict(kind="stencil_3d", grid=(nx, ny, nz), points=points, seed=seed,
                    drop_rate=drop_rate, drop_block=drop_block,
                    offband_row_frac=offband_row_frac, offband_per_row=offband_per_row,
                    offband_poisson=offband_poisson))


def paper_stencil(n: int, dim: int, *, seed: int = 0) -> CSR:
    """The stencil matrices of the paper's stencil experiments (Sec. 6.3): full
    diagonals j = i, i +- 1 (1D), also i +- n_x with n_x = floor(sqrt n) (2D),
    also i +- n_x^2 with n_x = floor(cbrt n) (3D), kept where 0 <= j < n.
    Values as in :func:`stencil_3d`."""
    offs = paper_stencil_offsets(n, dim)
    i = np.arange(n, dtype=np.int64)
    cols = i[:, None] + np.array(offs, dtype=np.int64)[None, :]
    mask = (cols >= 0) & (cols < n)
    keys = (i[:, None] * n + cols)[mask]
    row_ptr, col = _from_sorted_keys(n, keys)
    val = _dominant_values(n, row_ptr, col, Rng(seed, 3))
    return CSR(n, row_ptr, col, val, dict(kind="paper_stencil", dim=dim, n=n, seed=seed))


def paper_stencil_offsets(n: int, dim: int) -> list[int]:
    """Offsets of the paper's 1D/2D/3D stencils (Sec. 6.3) for n rows."""
    if dim == 1:
        return [-1, 0, 1]
    if dim == 2:
        nx = int(np.floor(np.sqrt(n)))
        while (nx + 1) ** 2 <= n:
            nx += 1
        while nx * nx > n:
            nx -= 1
        return sorted({-nx, -1, 0, 1, nx})
    if dim == 3:
        nx = int(round(n ** (1.0 / 3.0)))
        while (nx + 1) ** 3 <= n:
            nx += 1
        while nx ** 3 > n:
            nx -= 1
        return sorted({-nx * nx, -nx, -1, 0, 1, nx, nx * nx})
    raise ValueError("dim must be 1, 2 or 3")


def dia_matrix(n: int, offsets, *, seed: int, zero_rate: float = 0.0,
               pad: float = float("nan")) -> tuple[np.ndarray, np.ndarray]:
    """A seeded matrix in DIA input layout (Sec. 3.3, Fig. 4): returns
    (offsets int32[nd], val float64[nd, n]) with val[d, i] = a(i, i + offsets[d])
    drawn U[-1, 1] without exact zeros, a random ``zero_rate`` share of them
    set to 0.0 (positions without an entry), and ``pad`` at the positions
    outside the matrix (which the format ignores)."""
    off = np.asarray(sorted(set(int(o) for o in offsets)), dtype=np.int32)
    nd = off.size
    rng = Rng(seed, 17)
    val = rng.uniform(nd * n, -1.0, 1.0).reshape(nd, n)
    val[val == 0.0] = 0.5
    if zero_rate > 0:
        val[rng.bernoulli(nd * n, zero_rate).reshape(nd, n)] = 0.0
    i = np.arange(n, dtype=np.int64)
    for k, o in enumerate(off.tolist()):
        out = (i + o < 0) | (i + o >= n)
        val[k, out] = pad
    return off, val


def _loguniform(rng: Rng, k: int, lo_exp: float = -3.0, hi_exp: float = 3.0) -> np.ndarray:
    mag = 10.0 ** rng.uniform(k, lo_exp, hi_exp)
    sign = np.where(rng.bernoulli(k, 0.5), -1.0, 1.0)
    return sign * mag


def scattered_diagonals(n: int, n_offsets: int = 19, offset_range: int = 20000,
                        present_frac: float = 0.6, block: int = 2048,
                        extra_poisson: float = 3.0, *, seed: int = 2) -> CSR:
    """``n_offsets`` distinct offsets drawn uniformly in [-offset_range,
    offset_range]; each is present (all in-range rows) in a random
    ``present_frac`` of the ``block``-row blocks.  Every row also gets
    Poisson(``extra_poisson``) uniform random columns.  Values have magnitude
    log-uniform in [1e-3, 1e3] and a random sign."""
    rng_off = Rng(seed, 1)
    rng_extra = Rng(seed, 2)
    rng_val = Rng(seed, 3)
    offs: list[int] = []
    while len(offs) < n_offsets:
        o = int(rng_off.integers(1, -offset_range, offset_range + 1)[0])
        if o not in offs:
            offs.append(o)
    offs.sort()
    nblk = (n + block - 1) // block
    i = np.arange(n, dtype=np.int64)
    blk = i // block
    cols = np.empty((n, len(offs)), dtype=np.int64)
    mask = np.empty((n, len(offs)), dtype=bool)
    for k, o in enumerate(offs):
        present = rng_off.bernoulli(nblk, present_frac)
        cols[:, k] = i + o
        mask[:, k] = present[blk] & (i + o >= 0) & (i + o < n)
    keys = (i[:, None] * n + cols)[mask]
    del cols, mask
    if extra_poisson > 0.0:
        cnt = rng_extra.poisson(n, extra_poisson)
        keys = _add_random_entries(n, keys, np.repeat(i, cnt), rng_extra)
    row_ptr, col = _from_sorted_keys(n, keys)
    del keys
    val = _loguniform(rng_val, int(row_ptr[-1]))
    return CSR(n, row_ptr, col, val,
               dict(kind="scattered_diagonals", n=n, offsets=offs, present_frac=present_frac,
                    block=block, extra_poisson=extra_poisson, seed=seed))


def uniform_vector(n: int, seed: int, stream: int = 7, lo: float = -1.0,
                   hi: float = 1.0) -> np.ndarray:
    return Rng(seed, stream).uniform(n, lo, hi)


def loguniform_vector(n: int, seed: int, stream: int = 7) -> np.ndarray:
    return _loguniform(Rng(seed, stream), n)


def example_matrix() -> CSR:
    """The 8x8, 20-nonzero example matrix of the paper (Fig. 1)."""
    dense = np.array([
        [1, 0, 2, 0, 0, 3, 0, 0],
        [0, 4, 0, 5, 0, 0, 6, 0],
        [0, 0, 7, 0, 8, 0, 0, 9],
        [0, 0, 0, 10, 0, 0, 0, 0],
        [11, 0, 0, 0, 12, 0, 13, 0],
        [0, 0, 0, 0, 0, 14, 0, 15],
        [0, 0, 16, 0, 0, 0, 17, 0],
        [18, 0, 0, 19, 0, 0, 0, 20]], dtype=np.float64)
    return from_dense(dense, dict(kind="example"))


def from_dense(dense: np.ndarray, meta: dict | None = None) -> CSR:
    n = dense.shape[0]
    rows, cols = np.nonzero(dense)
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, row_ptr, cols.astype(np.int32), dense[rows, cols].astype(np.float64),
               meta or {})


def random_sparse(n: int, density: float, *, seed: int, diag_bias: float = 0.0) -> CSR:
    """Tiny random matrices for brute-force tests: entry (i, j) is stored with
    probability ``density`` (plus ``diag_bias`` on |i-j| <= 2); values
    U[-1, 1] without exact zeros."""
    rng = Rng(seed, 11)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    p = np.full((n, n), density) + diag_bias * (np.abs(i - j) <= 2)
    keep = rng.unit(n * n).reshape(n, n) < p
    vals = rng.uniform(n * n, -1.0, 1.0).reshape(n, n)
    vals[vals == 0.0] = 0.5
    dense = np.where(keep, vals, 0.0)
    return from_dense(dense, dict(kind="random_sparse", n=n, density=density, seed=seed))


# ---------------------------------------------------------------------------
# The named workloads
# ---------------------------------------------------------------------------

def _cache_dir() -> str | None:
    d = os.environ.get("MHDC_SYNTH_CACHE")
    if d is None:
        d = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                         ".synth_cache")
    if d in ("", "0", "off"):
        return None
    return d


def _cached(tag: str, make):
    d = _cache_dir()
    if d is None:
        return make()
    h = hashlib.sha1(tag.encode()).hexdigest()[:16]
    path = os.path.join(d, f"{h}.npz")
    if os.path.exists(path):
        try:
            z = np.load(path, allow_pickle=False)
            return CSR(int(z["n"]), z["row_ptr"], z["col"], z["val"], dict(cached=tag))
        except Exception:
            pass
    A = make()
    try:
        os.makedirs(d, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, n=A.n, row_ptr=A.row_ptr, col=A.col, val=A.val)
        os.replace(tmp, path)
    except OSError:
        pass
    return A


def config_matrix(name: str, scale: float = 1.0) -> CSR:
    """The named synthetic workloads.

    * ``"stencil7_32"``: 7-point FDM stencil on 32^3 (32,768 rows), seed 0.
    * ``"stencil27_128"``: 27-point stencil on 128^3, each off-centre offset
      dropped in a random 30% of 4096-row blocks, 2 random off-band entries in
      1% of the rows, seed 1.
    * ``"scattered_4m"``: 4,194,304 rows, 19 offsets in [-20000, 20000]
      present in 60% of 2048-row blocks, Poisson(3) random entries per row,
      log-uniform values, seed 2.

    ``scale`` < 1 shrinks the grid / row count for quick tests (same recipe).
    """
    if name == "stencil7_32":
        e = max(4, int(round(32 * scale)))
        return _cached(f"s7:{e}", lambda: stencil_3d(e, e, e, 7, seed=0))
    if name == "stencil27_128":
        e = max(4, int(round(128 * scale)))
        return _cached(f"s27:{e}", lambda: stencil_3d(
            e, e, e, 27, seed=1, drop_rate=0.3, drop_block=4096,
            offband_row_frac=0.01, offband_per_row=2))
    if name == "scattered_4m":
        n = max(4096, int(round(4194304 * scale)))
        rng = max(16, int(round(20000 * min(1.0, scale ** 0.5))))
        return _cached(f"sc:{n}:{rng}", lambda: scattered_diagonals(
            n, 19, rng, 0.6, 2048, 3.0, seed=2))
    raise KeyError(name)


def batch_matrices(count: int = 64, lo: int = 16, hi: int = 96, *, seed: int = 3) -> list[CSR]:
    """``count`` stencil matrices with grid edges uniform in {lo..hi}, 7- or
    27-point by a fair coin, values as :func:`stencil_3d`."""
    rng = Rng(seed, 21)
    edges = rng.integers(3 * count, lo, hi + 1).reshape(count, 3)
    kind = rng.bernoulli(count, 0.5)
    mats = []
    for m in range(count):
        nx, ny, nz = (int(v) for v in edges[m])
        pts = 27 if kind[m] else 7
        mats.append(_cached(f"b:{nx}:{ny}:{nz}:{pts}:{seed * 1000 + m}",
                            lambda nx=nx, ny=ny, nz=nz, pts=pts, sd=seed * 1000 + m:
                            stencil_3d(nx, ny, nz, pts, seed=sd)))
    return mats


def family_params(idx: int, *, base_seed: int = 1000, max_dim: int = 160,
                  min_dim: int = 32) -> dict:
    """Parameters of member ``idx`` of the selector's matrix family: 7/13/27
    points, grid dims in [min_dim, max_dim], block dropout in [0, 0.7],
    Poisson off-band density in [0, 5] per row, FP64 or FP32 values."""
    rng = Rng(base_seed + idx, 31)
    pts = (7, 13, 27)[int(rng.integers(1, 0, 3)[0])]
    dims = [int(v) for v in rng.integers(3, min_dim, max_dim + 1)]
    drop = float(rng.uniform(1, 0.0, 0.7)[0])
    dblk = (256, 1024, 4096)[int(rng.integers(1, 0, 3)[0])]
    off = float(rng.uniform(1, 0.0, 5.0)[0])
    f32 = bool(rng.bernoulli(1, 0.5)[0])
    return dict(points=pts, dims=dims, drop_rate=drop, drop_block=dblk,
                offband_poisson=off, value_dtype="f32" if f32 else "f64",
                seed=base_seed + idx)


def family_matrix(p: dict) -> CSR:
    nx, ny, nz = p["dims"]
    return stencil_3d(nx, ny, nz, p["points"], seed=p["seed"], drop_rate=p["drop_rate"],
                      drop_block=p["drop_block"], offband_poisson=p["offband_poisson"])
