"""Spatially varying blur: Theta = Psi* H Psi, its probe construction and its K-sparse
thresholding for a PSF that varies from image row to image row, in float64.

Paper passages followed:
  * Sec. 3.1, Def. "Blurring operators": (H u)(x) = int K(x, y) u(y) dy, with K(., y) the
    PSF at the location y; the class A(M, f) asks for PSFs that vary smoothly with y.
  * Sec. 3.5 (illustration, Fig. 1): a Gaussian PSF whose width grows linearly with y.
  * Sec. 3.4, Eq. matrixH: Theta[lam, mu] = <psi_lam, H psi_mu>; for a general operator the
    matrix is obtained by blurring wavelets and decomposing the result.
  * Sec. 3.7, Eq. naivethresholding / cleverthreshold: keep the K entries of largest
    |sigma_mu Theta[lam, mu]|, sigma_mu = 2^{s_b} for mu in subband b (level s_b), or 1.

Readings taken where the paper is silent:
  * Discrete operator: psfs[i] (odd kh x kw, centre at the origin) is the PSF with which the
    input pixels of image row i spread, on the torus:
        (H u)[(i + a) mod R, (j + b) mod C] += psfs[i][a + kh//2, b + kw//2] u[i, j].
    With one PSF for every row this is the convolution of oracle.blur.
  * Such an H commutes with horizontal translations, so Theta is circulant along the
    column axis inside every pair of subbands (a, b): Theta[(a, py, px), (b, qy, qx)]
    depends on (a, py, b, qy) and on one horizontal tap offset ox:
        column form (s_a <= s_b, r = 2^{s_b - s_a}): px = ox + r qx (mod C_a), |b| taken
            over the C_b positions qx of the input row;
        row form    (s_a >  s_b, r = 2^{s_a - s_b}): qx = ox + r px (mod C_b), over the
            C_a positions px of the output row.
    A tap is therefore (a, py, b, qy, ox) and carries the C_b (column form) or C_a (row
    form) entries of its horizontal diagonal. The column probe of input row (b, qy) is
    Psi* H psi_{b, qy, 0}; the row probe of output row (a, py) is Psi* H^T psi_{a, py, 0}.
    (theta_columns, which probes every column, is the plain definition these are pinned to.)
  * Thresholding keeps or drops whole taps: taps ranked by score (descending), ties broken by
    (a, py, b, qy, ox) ascending, accumulated while the running entry count stays <= K.
    A tap with |v| <= 1e-14 max|v| is a numerical zero and is never kept.
  * Preconditioner classes: Theta_K commutes with horizontal translations by 2^J pixels, so
    the diagonals of M = Theta_K^T Theta_K and of M^2 are periodic along every row of
    subband b with period R_b = 2^{J - s_b}; they are evaluated on one coordinate per class
    (b, qy, qx mod R_b), stored subband after subband, row-major in (qy, qx mod R_b).

TEST INFRASTRUCTURE: only tests, smoke() and the bench CPU baseline use this module.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .wavelet import Subband, dwt2, idwt2, layout

ZERO_REL = 1e-14


# ---------------------------------------------------------------------------------------
# The operator (Sec. 3.1)
# ---------------------------------------------------------------------------------------

def _check(psfs: np.ndarray, n_rows: int) -> tuple[int, int]:
    psfs = np.asarray(psfs)
    if psfs.ndim != 3 or psfs.shape[0] != n_rows:
        raise ValueError("psfs must be [n_rows, kh, kw]")
    kh, kw = psfs.shape[1:]
    if kh % 2 == 0 or kw % 2 == 0:
        raise ValueError("PSF sides must be odd")
    return kh, kw


def apply_H(u: np.ndarray, psfs: np.ndarray) -> np.ndarray:
    """H u: every nonzero input pixel spreads with the PSF of its row (zero pixels add
    nothing, so only the nonzeros are visited)."""
    u = np.asarray(u, dtype=np.float64)
    R, C = u.shape
    kh, kw = _check(psfs, R)
    ys, xs = np.nonzero(u)
    vals = u[ys, xs]
    out = np.zeros((R, C))
    for a in range(kh):
        ty = (ys + a - kh // 2) % R
        for b in range(kw):
            # for fixed (a, b) the targets are distinct, so a fancy-index add is exact
            out[ty, (xs + b - kw // 2) % C] += psfs[ys, a, b] * vals
    return out


def apply_Ht(v: np.ndarray, psfs: np.ndarray) -> np.ndarray:
    """H^T v: (H^T v)[i, j] = sum_{a, b} psfs[i][a, b] v[(i + a - kh//2), (j + b - kw//2)];
    only the rows within reach of a nonzero row of v are evaluated (the others are 0)."""
    v = np.asarray(v, dtype=np.float64)
    R, C = v.shape
    kh, kw = _check(psfs, R)
    nz = np.nonzero(np.any(v != 0.0, axis=1))[0]
    rows = np.unique(((nz[:, None] - (np.arange(kh) - kh // 2)[None, :]) % R).ravel())
    out = np.zeros((R, C))
    acc = np.zeros((len(rows), C))
    for a in range(kh):
        block = v[(rows + a - kh // 2) % R]
        for b in range(kw):
            # np.roll(block, -d, axis=1)[:, j] = block[:, (j + d) mod C]
            acc += psfs[rows, a, b][:, None] * np.roll(block, -(b - kw // 2), axis=1)
    out[rows] = acc
    return out


def H_dense(psfs: np.ndarray, n_rows: int, n_cols: int) -> np.ndarray:
    """The N x N matrix of H, column y = H e_y (tiny sizes only)."""
    N = n_rows * n_cols
    Hm = np.zeros((N, N))
    for y in range(N):
        e = np.zeros(N)
        e[y] = 1.0
        Hm[:, y] = apply_H(e.reshape(n_rows, n_cols), psfs).ravel()
    return Hm


def theta_columns(psfs: np.ndarray, n_rows: int, n_cols: int, wavelet: str, levels: int) -> np.ndarray:
    """Theta, every column probed (Sec. 3.4): column mu = Psi* H Psi e_mu (tiny sizes only)."""
    N = n_rows * n_cols
    T = np.zeros((N, N))
    for mu in range(N):
        e = np.zeros(N)
        e[mu] = 1.0
        T[:, mu] = dwt2(apply_H(idwt2(e, n_rows, n_cols, wavelet, levels), psfs), wavelet, levels)
    return T


# ---------------------------------------------------------------------------------------
# Probes: one per input row (column form) and one per output row (row form)
# ---------------------------------------------------------------------------------------

def _unit_wavelet(sb: Subband, row: int, n_rows: int, n_cols: int, wavelet: str, levels: int) -> np.ndarray:
    e = np.zeros(n_rows * n_cols)
    e[sb.offset + row * sb.cols] = 1.0
    return idwt2(e, n_rows, n_cols, wavelet, levels)


def column_probe(psfs, n_rows, n_cols, wavelet, levels, b_index, qy):
    """Psi* H psi_{b, qy, 0}."""
    sb = layout(n_rows, n_cols, levels)[b_index]
    return dwt2(apply_H(_unit_wavelet(sb, qy, n_rows, n_cols, wavelet, levels), psfs), wavelet, levels)


def row_probe(psfs, n_rows, n_cols, wavelet, levels, a_index, py):
    """Psi* H^T psi_{a, py, 0}."""
    sa = layout(n_rows, n_cols, levels)[a_index]
    return dwt2(apply_Ht(_unit_wavelet(sa, py, n_rows, n_cols, wavelet, levels), psfs), wavelet, levels)


@dataclass
class VTaps:
    """Flat list of distinct taps (one per horizontal diagonal of every row pair)."""
    a: np.ndarray      # output subband
    py: np.ndarray     # output row in a
    b: np.ndarray      # input subband
    qy: np.ndarray     # input row in b
    ox: np.ndarray     # horizontal tap offset
    v: np.ndarray      # value
    m: np.ndarray      # multiplicity (entries carrying the value)

    def __len__(self):
        return len(self.v)

    def subset(self, mask) -> "VTaps":
        return VTaps(*(z[mask] for z in (self.a, self.py, self.b, self.qy, self.ox, self.v, self.m)))


def _probe_taps(kind: int, psfs, n_rows, n_cols, wavelet, levels, sub, row):
    """The taps one probe gives, exact zeros dropped (they can never be kept):
    kind 0: column probe of input row (sub, row) -> pairs (a, b = sub) with s_a <= s_b;
    kind 1: row probe of output row (sub, row)   -> pairs (a = sub, b) with s_b < s_a."""
    lay = layout(n_rows, n_cols, levels)
    fixed = lay[sub]
    vec = (column_probe if kind == 0 else row_probe)(psfs, n_rows, n_cols, wavelet, levels, sub, row)
    out = []
    for o in lay:
        if (kind == 0 and o.level > fixed.level) or (kind == 1 and o.level >= fixed.level):
            continue
        blk = vec[o.offset:o.offset + o.size].reshape(o.rows, o.cols)
        r, c = np.nonzero(blk)
        if len(r) == 0:
            continue
        n = len(r)
        if kind == 0:       # output a = o, rows r; input (sub, row)
            a, py, b, qy, m = np.full(n, o.index), r, np.full(n, sub), np.full(n, row), fixed.cols
        else:               # output (sub, row); input b = o, rows r
            a, py, b, qy, m = np.full(n, sub), np.full(n, row), np.full(n, o.index), r, fixed.cols
        out.append((a, py, b, qy, c, blk[r, c], np.full(n, m, dtype=np.int64)))
    if not out:
        return tuple(np.zeros(0, dtype=np.int64) for _ in range(5)) + (np.zeros(0), np.zeros(0, dtype=np.int64))
    return tuple(np.concatenate(z) for z in zip(*out))


_WORKER_OP = None


def _worker_init(psfs, n_rows, n_cols, wavelet, levels):
    global _WORKER_OP
    _WORKER_OP = (psfs, n_rows, n_cols, wavelet, levels)


def _worker_probe(job):
    kind, sub, row = job
    return _probe_taps(kind, *_WORKER_OP, sub, row)


def all_taps(psfs: np.ndarray, n_rows: int, n_cols: int, wavelet: str, levels: int, workers: int = 1) -> VTaps:
    """Every nonzero tap of Theta: column probes give the pairs with s_a <= s_b, row probes
    the pairs with s_a > s_b (multiplicity: the columns of the coarser subband). workers > 1
    only spreads the independent probes over that many spawned processes."""
    lay = layout(n_rows, n_cols, levels)
    jobs = [(0, b.index, q) for b in lay for q in range(b.rows)]
    jobs += [(1, a.index, q) for a in lay if a.level > 1 for q in range(a.rows)]
    common = (psfs, n_rows, n_cols, wavelet, levels)
    if workers <= 1:
        res = [_probe_taps(k, *common, s, q) for k, s, q in jobs]
    else:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                 initializer=_worker_init, initargs=common) as pool:
            res = list(pool.map(_worker_probe, jobs, chunksize=16))
    cols = [np.concatenate([r[i] for r in res]) for i in range(7)]
    return VTaps(*cols)


# ---------------------------------------------------------------------------------------
# Sec. 3.7 thresholding over taps
# ---------------------------------------------------------------------------------------

def tap_scores(t: VTaps, lay: list, rule: str) -> np.ndarray:
    """|sigma_b v| with sigma_b = 2^{s_b} (weighted rule) or 1 (naive rule)."""
    if rule == "weighted":
        lev = np.array([s.level for s in lay], dtype=np.float64)
        return np.abs(2.0 ** lev[t.b] * t.v)
    if rule == "naive":
        return np.abs(t.v)
    raise ValueError(rule)


def select_taps(t: VTaps, lay: list, K: int, rule: str = "weighted") -> np.ndarray:
    """Keep-mask: the longest prefix of the (score desc, a, py, b, qy, ox asc) order whose
    total multiplicity is <= K, numerical zeros excluded."""
    vmax = np.abs(t.v).max() if len(t) else 0.0
    idx = np.nonzero(np.abs(t.v) > ZERO_REL * vmax)[0]
    score = tap_scores(t, lay, rule)
    # np.lexsort: the LAST key is the primary key
    order = idx[np.lexsort((t.ox[idx], t.qy[idx], t.b[idx], t.py[idx], t.a[idx], -score[idx]))]
    n_keep = int(np.searchsorted(np.cumsum(t.m[order]), K, side="right"))
    keep = np.zeros(len(t), dtype=bool)
    keep[order[:n_keep]] = True
    return keep


def tap_entries(t: VTaps, lay: list):
    """(rows, cols, vals) of every entry carried by the taps (the two forms above)."""
    rows, cols, vals = [], [], []
    if len(t) == 0:
        return np.zeros(0, int), np.zeros(0, int), np.zeros(0)
    pairs = np.unique(np.stack([t.a, t.b], axis=1), axis=0)
    for ai, bi in pairs:
        a, b = lay[ai], lay[bi]
        sel = (t.a == ai) & (t.b == bi)
        py, qy, ox, v = t.py[sel], t.qy[sel], t.ox[sel], t.v[sel]
        if a.level <= b.level:
            r = 1 << (b.level - a.level)
            qx = np.arange(b.cols)[None, :]
            px = (ox[:, None] + r * qx) % a.cols
            qx = np.broadcast_to(qx, px.shape)
        else:
            r = 1 << (a.level - b.level)
            px = np.arange(a.cols)[None, :]
            qx = (ox[:, None] + r * px) % b.cols
            px = np.broadcast_to(px, qx.shape)
        rows.append((a.offset + py[:, None] * a.cols + px).ravel())
        cols.append((b.offset + qy[:, None] * b.cols + qx).ravel())
        vals.append(np.broadcast_to(v[:, None], px.shape).ravel())
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


def theta_sparse(t: VTaps, lay: list, N: int) -> sp.csr_matrix:
    r, c, v = tap_entries(t, lay)
    return sp.csr_matrix((v, (r, c)), shape=(N, N))


@dataclass
class VThetaK:
    n_rows: int
    n_cols: int
    wavelet: str
    levels: int
    lay: list
    taps: VTaps         # kept taps only
    K_requested: int
    K_eff: int
    n_candidates: int   # nonzero taps before thresholding
    mat: sp.csr_matrix
    matT: sp.csr_matrix


def build_varying_theta(psfs: np.ndarray, n_rows: int, n_cols: int, wavelet: str, levels: int,
                        K: int, rule: str = "weighted", workers: int = 1) -> VThetaK:
    """Probes (one per row of every subband) + Sec. 3.7 thresholding -> Theta_K."""
    if K < 0:
        raise ValueError("K must be >= 0")
    t = all_taps(psfs, n_rows, n_cols, wavelet, levels, workers=workers)
    lay = layout(n_rows, n_cols, levels)
    keep = select_taps(t, lay, K, rule)
    kt = t.subset(keep)
    mat = theta_sparse(kt, lay, n_rows * n_cols)
    vmax = np.abs(t.v).max() if len(t) else 0.0
    ncand = int(np.count_nonzero(np.abs(t.v) > ZERO_REL * vmax))
    return VThetaK(n_rows, n_cols, wavelet, levels, lay, kt, int(K), int(kt.m.sum()), ncand, mat, mat.T.tocsr())


# ---------------------------------------------------------------------------------------
# Preconditioner classes (Sec. 4.2, 4.3 on this operator)
# ---------------------------------------------------------------------------------------

def class_periods(lay: list, levels: int) -> list:
    """R_b = 2^{J - s_b}: period of the diagonals of M along the rows of subband b."""
    return [1 << (levels - b.level) for b in lay]


def class_offsets(lay: list, periods: list) -> np.ndarray:
    sizes = np.array([b.rows * periods[b.index] for b in lay])
    return np.concatenate([[0], np.cumsum(sizes)])


def diagonal_tables(mat, matT, lay, periods) -> tuple[np.ndarray, np.ndarray]:
    """M_ii and (M^2)_ii per class (b, qy, qx mod R_b), representative column qx < R_b."""
    csc = mat.tocsc()
    offs = class_offsets(lay, periods)
    Md = np.zeros(offs[-1])
    M2d = np.zeros(offs[-1])
    for b in lay:
        R = periods[b.index]
        for qy in range(b.rows):
            for px in range(R):
                i = b.offset + qy * b.cols + px
                v = csc[:, [i]]
                w = matT @ v
                t = offs[b.index] + qy * R + px
                Md[t] = float(v.multiply(v).sum())
                M2d[t] = float(w.multiply(w).sum())
    return Md, M2d


def expand(table: np.ndarray, lay, periods) -> np.ndarray:
    """Class table -> N-vector in planar order."""
    offs = class_offsets(lay, periods)
    out = []
    for b in lay:
        R = periods[b.index]
        tab = table[offs[b.index]:offs[b.index + 1]].reshape(b.rows, R)
        out.append(tab[:, np.arange(b.cols) % R].ravel())
    return np.concatenate(out)
