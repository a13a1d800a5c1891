"""Theta = Psi* H Psi for a periodic convolution, its probe construction and its K-sparse
thresholding, in float64.

Paper passages followed:
  * Eq. (matrixH), Sec. 3.4: Theta = Psi* H Psi, rows indexed by outputs. Entry
    Theta[lam, mu] = <psi_lam, H psi_mu>. (Eq. definition_theta in Sec. 3.2 writes the
    transposed pairing <H psi_lam, psi_mu>; the two agree for symmetric PSFs. The Sec. 3.4
    matrix reading is the one for which 1/2||Theta x - x0||^2 = 1/2||H Psi x - u0||^2, the
    identity of Eq. l1problemTheta, so it is the one used.)
  * Def. "Rectangular circulant matrices" and Thm 3 (Sec. 3.6): every block Theta_{a,b}
    between two subbands is circulant with shifts 2^{|s_a - s_b|}.
  * Algorithm 2 (Sec. 3.6): one probe per subband b: psi_b = wavelet at position 0; blur it
    with H (column probe) and H^T (row probe); one forward DWT each. Blocks whose output
    subband is finer than or as fine as the input take column taps, blocks whose output is
    coarser take row taps.
  * Eq. naivethresholding / cleverthreshold (Sec. 3.7): keep the K entries of largest
    |sigma_mu Theta[lam, mu]|, sigma_mu = 2^{-k} for mu at scale k (k counted from the
    coarsest scale), i.e. sigma proportional to 2^{s_b} with s_b the input subband level;
    sigma = 1 for the naive rule.

Readings taken where the paper is silent:
  * Entries of one circulant block that share a tap are equal, so the thresholding keeps or
    drops whole taps. Taps are ranked by score (descending), ties broken by (a, b, oy, ox)
    ascending, and accumulated while the running entry count stays <= K; the first tap that
    would exceed K ends the selection ("at most K non zero entries", Sec. 1.3).
  * A tap with |v| <= 1e-14 * max|v| is a numerical zero and is never kept.

TEST INFRASTRUCTURE: only tests, smoke() and the bench CPU baseline use this module.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .blur import conv_adjoint, conv_matrix, conv_periodic
from .wavelet import Subband, dwt2, dwt_matrix, idwt2, layout, synthesis_1d, wavelet_filters

ZERO_REL = 1e-14


# ---------------------------------------------------------------------------------------
# Dense brute force (tiny sizes)
# ---------------------------------------------------------------------------------------

def theta_dense(n_rows: int, n_cols: int, psf: np.ndarray, wavelet: str, levels: int) -> np.ndarray:
    """Theta = D H D^T with D = Psi* (Eq. matrixH), every matrix built from unit vectors."""
    D = dwt_matrix(n_rows, n_cols, wavelet, levels)
    Hm = conv_matrix(n_rows, n_cols, psf)
    return D @ Hm @ D.T


# ---------------------------------------------------------------------------------------
# Circulant block index rule (Def. rectangular circulant matrices)
# ---------------------------------------------------------------------------------------

def block_tap_index(n_out: int, n_in: int) -> np.ndarray:
    """1-D index map M[p, q] into the tap vector of one circulant block.

    n_out >= n_in (output finer or equal, ratio r = n_out/n_in, tap vector of length n_out,
    column form):  M[p, q] = (p - r q) mod n_out.
    n_out <  n_in (output coarser, r = n_in/n_out, tap vector of length n_in, row form):
                   M[p, q] = (q - r p) mod n_in.
    The paper's 4 x 8 example has A[l, :] = tau_{2l}(a), i.e. A[l, m] = a[m - 2l].
    """
    p = np.arange(n_out)[:, None]
    q = np.arange(n_in)[None, :]
    if n_out >= n_in:
        r = n_out // n_in
        return (p - r * q) % n_out
    r = n_in // n_out
    return (q - r * p) % n_in


# ---------------------------------------------------------------------------------------
# Algorithm 2: probes and taps
# ---------------------------------------------------------------------------------------

@dataclass
class Probes:
    n_rows: int
    n_cols: int
    wavelet: str
    levels: int
    lay: list
    col: list        # col[b] = Psi* H psi_{b,0}   (N-vector)
    row: list        # row[b] = Psi* H^T psi_{b,0} (N-vector)


def probe(psf: np.ndarray, n_rows: int, n_cols: int, wavelet: str, levels: int, offset: int):
    """(Psi* H psi, Psi* H^T psi) for psi the wavelet of coefficient `offset` (Algorithm 2)."""
    e = np.zeros(n_rows * n_cols)
    e[offset] = 1.0
    psi = idwt2(e, n_rows, n_cols, wavelet, levels)
    return (dwt2(conv_periodic(psi, psf), wavelet, levels),
            dwt2(conv_adjoint(psi, psf), wavelet, levels))


def compute_probes(psf: np.ndarray, n_rows: int, n_cols: int, wavelet: str, levels: int,
                   pool=None) -> Probes:
    """Algorithm 2, probe stage: for every subband b, blur the wavelet psi_{b,0} (the
    coefficient at position (0,0) of b) with H and H^T and take one forward DWT of each.
    `pool` (an executor) only spreads the independent probes over processes."""
    lay = layout(n_rows, n_cols, levels)
    args = [(psf, n_rows, n_cols, wavelet, levels, b.offset) for b in lay]
    if pool is None:
        res = [probe(*a) for a in args]
    else:
        res = list(pool.map(probe, *zip(*args)))
    return Probes(n_rows, n_cols, wavelet, levels, lay, [c for c, _ in res], [r for _, r in res])


def pair_taps(pr: Probes, a: Subband, b: Subband) -> tuple[np.ndarray, int, bool]:
    """Tap array of block (a, b), its multiplicity and whether it is in column form.

    Column form (s_a <= s_b): taps = col[b] restricted to subband a, shape (R_a, C_a),
    multiplicity = |b|.  Row form (s_a > s_b): taps = row[a] restricted to subband b,
    shape (R_b, C_b), multiplicity = |a|.
    """
    if a.level <= b.level:
        v = pr.col[b.index][a.offset:a.offset + a.size].reshape(a.rows, a.cols)
        return v, b.size, True
    v = pr.row[a.index][b.offset:b.offset + b.size].reshape(b.rows, b.cols)
    return v, a.size, False


@dataclass
class Taps:
    """Flat list of distinct taps (one per circulant diagonal of every block)."""
    a: np.ndarray      # output subband index
    b: np.ndarray      # input subband index
    oy: np.ndarray     # tap offset (row) inside its tap array
    ox: np.ndarray     # tap offset (col)
    v: np.ndarray      # value
    m: np.ndarray      # multiplicity (entries of Theta carrying this value)

    def __len__(self):
        return len(self.v)

    def subset(self, mask) -> "Taps":
        return Taps(self.a[mask], self.b[mask], self.oy[mask], self.ox[mask], self.v[mask], self.m[mask])


def all_taps(pr: Probes) -> Taps:
    """Every distinct tap of Theta (the full operator, before thresholding)."""
    A, B, OY, OX, V, M = [], [], [], [], [], []
    for a in pr.lay:
        for b in pr.lay:
            v, mult, _ = pair_taps(pr, a, b)
            oy, ox = np.meshgrid(np.arange(v.shape[0]), np.arange(v.shape[1]), indexing="ij")
            A.append(np.full(v.size, a.index))
            B.append(np.full(v.size, b.index))
            OY.append(oy.ravel())
            OX.append(ox.ravel())
            V.append(v.ravel())
            M.append(np.full(v.size, mult, dtype=np.int64))
    return Taps(*(np.concatenate(z) for z in (A, B, OY, OX, V, M)))


# ---------------------------------------------------------------------------------------
# Sec. 3.7 thresholding
# ---------------------------------------------------------------------------------------

def tap_scores(t: Taps, lay: list, rule: str) -> np.ndarray:
    """|sigma_b v| with sigma_b = 2^{s_b} (weighted rule) or 1 (naive rule)."""
    if rule == "weighted":
        lev = np.array([s.level for s in lay], dtype=np.float64)
        sigma = 2.0 ** lev[t.b]
    elif rule == "naive":
        sigma = np.ones(len(t))
    else:
        raise ValueError(rule)
    return np.abs(sigma * t.v)


def select_taps(t: Taps, lay: list, K: int, rule: str = "weighted") -> np.ndarray:
    """Boolean keep-mask over taps: the longest prefix of the (score desc, a, b, oy, ox asc)
    order whose total multiplicity is <= K, numerical zeros excluded."""
    vmax = np.abs(t.v).max() if len(t) else 0.0
    nonzero = np.abs(t.v) > ZERO_REL * vmax
    score = tap_scores(t, lay, rule)
    idx = np.nonzero(nonzero)[0]
    # np.lexsort: the LAST key is the primary key
    order = idx[np.lexsort((t.ox[idx], t.oy[idx], t.b[idx], t.a[idx], -score[idx]))]
    csum = np.cumsum(t.m[order])
    n_keep = int(np.searchsorted(csum, K, side="right"))
    keep = np.zeros(len(t), dtype=bool)
    keep[order[:n_keep]] = True
    return keep


# ---------------------------------------------------------------------------------------
# Expansion of taps into entries of Theta_K
# ---------------------------------------------------------------------------------------

def tap_entries(t: Taps, lay: list):
    """(rows, cols, vals) of every entry carried by the taps, from the circulant rule.

    Column form (s_a <= s_b, r = 2^{s_b - s_a}): entry ((a, p), (b, q)) for p = o + r q.
    Row form    (s_a >  s_b, r = 2^{s_a - s_b}): entry ((a, p), (b, q)) for q = o + r p.
    Indices are taken modulo the subband sides.
    """
    rows, cols, vals = [], [], []
    pairs = np.unique(np.stack([t.a, t.b], axis=1), axis=0) if len(t) else np.zeros((0, 2), int)
    for ai, bi in pairs:
        a, b = lay[ai], lay[bi]
        sel = (t.a == ai) & (t.b == bi)
        oy, ox, v = t.oy[sel], t.ox[sel], t.v[sel]
        if a.level <= b.level:
            r = 1 << (b.level - a.level)
            qy, qx = np.meshgrid(np.arange(b.rows), np.arange(b.cols), indexing="ij")
            qy, qx = qy.ravel(), qx.ravel()
            py = (oy[:, None] + r * qy[None, :]) % a.rows
            px = (ox[:, None] + r * qx[None, :]) % a.cols
            Q = np.broadcast_to(b.offset + qy * b.cols + qx, py.shape)
            Pp = a.offset + py * a.cols + px
        else:
            r = 1 << (a.level - b.level)
            py_, px_ = np.meshgrid(np.arange(a.rows), np.arange(a.cols), indexing="ij")
            py_, px_ = py_.ravel(), px_.ravel()
            qy = (oy[:, None] + r * py_[None, :]) % b.rows
            qx = (ox[:, None] + r * px_[None, :]) % b.cols
            Q = b.offset + qy * b.cols + qx
            Pp = np.broadcast_to(a.offset + py_ * a.cols + px_, Q.shape)
        rows.append(Pp.ravel())
        cols.append(Q.ravel())
        vals.append(np.broadcast_to(v[:, None], Q.shape).ravel())
    if not rows:
        return np.zeros(0, int), np.zeros(0, int), np.zeros(0)
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


def theta_sparse(t: Taps, lay: list, N: int) -> sp.csr_matrix:
    """Theta_K as a CSR matrix (rows = outputs)."""
    r, c, v = tap_entries(t, lay)
    return sp.csr_matrix((v, (r, c)), shape=(N, N))


@dataclass
class ThetaK:
    """The thresholded operator and what it was built from."""
    n_rows: int
    n_cols: int
    wavelet: str
    levels: int
    lay: list
    taps: Taps          # kept taps only
    K_requested: int
    K_eff: int
    mat: sp.csr_matrix  # Theta_K
    matT: sp.csr_matrix  # Theta_K^T


def build_theta(psf: np.ndarray, n_rows: int, n_cols: int, wavelet: str, levels: int,
                K: int, rule: str = "weighted", pool=None) -> ThetaK:
    """Algorithm 2 probes + Sec. 3.7 thresholding -> Theta_K."""
    if K < 0:
        raise ValueError("K must be >= 0")
    pr = compute_probes(psf, n_rows, n_cols, wavelet, levels, pool=pool)
    t = all_taps(pr)
    keep = select_taps(t, pr.lay, K, rule)
    kt = t.subset(keep)
    N = n_rows * n_cols
    mat = theta_sparse(kt, pr.lay, N)
    return ThetaK(n_rows, n_cols, wavelet, levels, pr.lay, kt, int(K), int(kt.m.sum()),
                  mat, mat.T.tocsr())


# ---------------------------------------------------------------------------------------
# Single entries at any size (separable wavelets)
# ---------------------------------------------------------------------------------------

def wavelet_1d(n: int, level: int, high: bool, pos: int, wavelet: str) -> np.ndarray:
    """The 1-D periodic synthesis function of length n of the coefficient `pos` at `level`:
    a unit coefficient synthesised once with g (high) or h, then with h down to level 0
    (the axis factor of a 2-D wavelet of oracle.wavelet's separable transform)."""
    h, g = wavelet_filters(wavelet)
    c = np.zeros(n >> level)
    c[pos] = 1.0
    for s in range(level, 0, -1):
        c = synthesis_1d(c[None, :], g if (s == level and high) else h, axis=1)[0]
    return c


def theta_entry(psf: np.ndarray, n_rows: int, n_cols: int, wavelet: str, levels: int,
                a: int, p: tuple, b: int, q: tuple) -> float:
    """Theta[(a, p), (b, q)] = <psi_{a,p}, H psi_{b,q}> (Eq. matrixH) for one entry.

    Both wavelets are outer products of 1-D functions, psi(y) = f_v(y_r) f_h(y_c), so with
    (H u)[i] = sum_d psf[d] u[i - d]:
        <psi_a, H psi_b> = sum_d psf[d] C_v(d_r) C_h(d_c),
        C(d) = sum_j f_a(j + d) f_b(j)   (periodic),
    a sum over the PSF support of products of two 1-D correlations."""
    lay = layout(n_rows, n_cols, levels)
    sa, sb = lay[a], lay[b]
    fav = wavelet_1d(n_rows, sa.level, sa.e[0] == 1, p[0], wavelet)
    fah = wavelet_1d(n_cols, sa.level, sa.e[1] == 1, p[1], wavelet)
    fbv = wavelet_1d(n_rows, sb.level, sb.e[0] == 1, q[0], wavelet)
    fbh = wavelet_1d(n_cols, sb.level, sb.e[1] == 1, q[1], wavelet)
    kh, kw = psf.shape
    # np.roll(f, -d)[j] = f[(j + d) mod n]
    Cv = np.array([np.dot(np.roll(fav, -d), fbv) for d in range(-(kh // 2), kh // 2 + 1)])
    Ch = np.array([np.dot(np.roll(fah, -d), fbh) for d in range(-(kw // 2), kw // 2 + 1)])
    return float(Cv @ psf @ Ch)
