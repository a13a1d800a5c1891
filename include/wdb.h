/*
 * wdb.h — C ABI of libwdb: wavelet-domain l1-l2 deblurring (Escande & Weiss, arXiv 1512.08401)
 * on one NVIDIA GB300 (sm_103a).
 *
 * The library solves
 *     min_x  E(x) = 1/2 || Theta_K x - x0 ||^2 + sum_i w_i |x_i|          (Eq. l1problemThetaApprox)
 * with x0 = Psi* u0 the wavelet coefficients of the observed image u0 (Sec. 1.3),
 * Theta_K the K-sparse approximation of Theta = Psi* H Psi (Eq. matrixH) of a periodic
 * convolution H, built by Algorithm 2 and thresholded by Eq. cleverthreshold, and the solver
 * is diagonally preconditioned FISTA (Algorithm 3, Sec. 4.2/4.3). The exact-operator
 * path (Algorithm 1 with the gradient computed by FFTs and wavelet transforms, Sec. 5.2)
 * runs on the same GPU for comparison.
 *
 * Conventions shared by every entry point
 *   - Images are row-major float (FP32) arrays of n_rows x n_cols pixels; both sides must be
 *     divisible by 2^levels. The domain is the torus (periodic boundaries, Sec. 2).
 *   - Wavelet coefficient vectors hold N = n_rows * n_cols floats in subband-planar order:
 *     the approximation A_J (n_rows/2^J x n_cols/2^J, row-major), then for s = J, J-1, ..., 1
 *     the detail subbands with orientation (e_y, e_x) = (0,1), (1,0), (1,1), each
 *     n_rows/2^s x n_cols/2^s row-major. Subband index 0 is A_J; 3J+1 subbands in all.
 *   - wavelet names "db1" ... "db10": orthogonal Daubechies filters with p vanishing
 *     moments (2p taps), minimum phase; "sym1" ... "sym10": the same filter magnitudes with
 *     the zeros chosen for the phase closest to linear (Symmlets; the paper's experiments use
 *     Symmlet 6, Sec. 5). Periodic separable 2-D transform (Sec. 2).
 *   - PSF: host FP64 array of kh x kw (odd sizes), row-major; element (kh/2, kw/2) is the
 *     origin; (H u)[i,j] = sum_{a,b} psf[a+kh/2][b+kw/2] u[i-a][j-b] (indices mod n).
 *   - Pointers named *_dev are device pointers owned by the caller; they must stay valid
 *     until the stream has finished the call's work. Pointers named *_host are host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Every call returns a wdb_status. Nothing is thrown across the ABI and nothing aborts.
 *     After an error, wdb_last_error() returns a one-line description (thread-local).
 *     Asynchronous CUDA errors surface as WDB_ECUDA at the next synchronising call.
 *   - A wdb_theta or wdb_fftop handle may be used by one stream at a time.
 */
#ifndef WDB_H
#define WDB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WDB_OK = 0,
    WDB_EINVAL = 1,        /* invalid argument (sizes, names, NULL pointers, ranges) */
    WDB_ENOMEM = 2,        /* device or host allocation failed */
    WDB_ECUDA = 3,         /* a CUDA runtime / cuFFT call failed */
    WDB_ENAN = 4,          /* a NaN or Inf appeared in the objective or the certificate */
    WDB_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    WDB_EDIVERGED = 6,     /* the objective grew by more than 1e6 x its first value */
    WDB_EUNSUPPORTED = 7,  /* valid but not supported (e.g. more than 64 subbands) */
    WDB_EIO = 8,           /* file could not be read or written, or has a bad format */
    WDB_EPLAN = 9          /* a tile plan broke one of its invariants (wdb_tile_plan_check) */
} wdb_status;

#define WDB_MAX_SUBBANDS 64
#define WDB_PRECOND_NONE 0
#define WDB_PRECOND_JACOBI 1   /* Eq. Jacobi_Precond: P = max(diag(Theta_K^T Theta_K), eps) */
#define WDB_PRECOND_SPAI 2     /* Eq. SPAI_Precond:  P_ii = (M^2)_ii / M_ii, M = Theta_K^T Theta_K */
#define WDB_RULE_WEIGHTED 0    /* Eq. cleverthreshold: score |2^{s_b} Theta[a,b]| */
#define WDB_RULE_NAIVE 1       /* Eq. naivethresholding: score |Theta[a,b]| */

typedef struct wdb_theta wdb_theta;   /* Theta_K and its preconditioners, library-owned */
typedef struct wdb_fftop wdb_fftop;   /* exact operator H Psi for the FFT path, library-owned */
typedef struct wdb_vtheta wdb_vtheta; /* Theta_K of a row-varying blur, library-owned */

/* Summary of a Theta_K handle. */
typedef struct {
    int n_rows, n_cols, levels, n_subbands;
    int wavelet_taps;           /* 2p */
    int rule;                   /* WDB_RULE_* used to select taps */
    long long K_requested;      /* K passed to wdb_build_theta */
    long long K_eff;            /* nonzero entries of Theta_K (<= K_requested) */
    long long n_taps;           /* distinct kept taps (one per circulant diagonal) */
    long long n_candidates;     /* distinct taps of the full Theta before thresholding */
    double theta_max_abs;       /* max |tap| of the full Theta */
    int phase_table_len;        /* 4^J: length of the per-phase-class preconditioner tables */
    double build_ms;            /* wall time of wdb_build_theta (device work included) */
    int plan_tuned;             /* 1: the FP32 kernels' plans were autotuned on this GPU */
    int plan_items[2];          /* work items of the FP32 plans of Theta_K and Theta_K^T */
    int plan_split_tiles[2];    /* tiles of those plans split over several CTAs */
    int plan_super_subbands[2]; /* subbands of those plans worked in 2 x 2 super tiles */
    int plan_groups[2];         /* groups of subbands worked together by those plans' items */
    int plan_smem_bytes[2];     /* dynamic shared memory per CTA of those plans (two staging buffers) */
    int plan_grid[2];           /* persistent CTAs those plans launch (SMs x resident CTAs per SM) */
} wdb_theta_info;

/* Parameters of one solve. Zero-initialise and set what you need. */
typedef struct {
    double lambda;              /* w_i = lambda for every coefficient when w_subband == NULL */
    const double* w_subband_host;  /* optional: n_subbands weights (Eq. def:G, w constant per subband) */
    int max_iters;              /* iteration cap (>= 1) */
    double tol;                 /* stop when gap/primal <= tol at a check; 0: run max_iters */
    int precond;                /* WDB_PRECOND_* */
    double jacobi_eps;          /* <= 0: 1e-6 * max_i M_ii */
    int check_every;            /* gap check period m (<= 0: 10) */
    const float* x_init_dev;    /* N floats or NULL (zero start) */
    int no_graph;               /* 1: launch kernels one by one instead of CUDA graphs */
    double target_objective;    /* > 0: also stop at the first k whose primal value at y^(k)
                                   is <= target (checked on the device every iteration) */
    int time_kernels;           /* 1: time one residual and one step launch per chunk with
                                   CUDA events (reported in the result) */
    int kkt_check;              /* 1: after the loop, check the returned x in FP64 on the device
                                   (wdb_theta_kkt; the kkt_* and *64 fields of the result) */
    int ista;                   /* 1: drop the momentum step, y^(k+1) = x^(k) (ISTA, the baseline
                                   of the paper's Sec. 5.3 comparison); 0: Algorithm 3 */
    int fused;                  /* 1: run each chunk of check_every iterations as one cooperative
                                   launch of the resident CTAs (kernel 1 and kernel 2 of every
                                   iteration separated by grid barriers); falls back to two
                                   launches per iteration for plans with split tiles */
    long long spin_limit;       /* fused loop: polls a grid barrier's wait makes before giving up
                                   with WDB_ETIMEOUT (<= 0: 2^23, well over a second) */
} wdb_solve_params;

typedef struct {
    int iters;                  /* iterations run (the k of the returned x^(k)) */
    double objective;           /* E(x) of the returned x, FP64 (Theta_K problem, or exact for the FFT path) */
    double primal, gap, rel_gap;/* duality-gap certificate of y^(k) at the last check (NaN if none) */
    long long support;          /* number of nonzero coefficients of x */
    double tau, L_hat;          /* step and Lipschitz estimate used */
    double solve_ms;            /* wall time of the call including the final synchronisation */
    double ms_k1, ms_k2;        /* time_kernels: mean duration of one residual launch (kernel 1;
                                   FFT path: IDWT+R2C+spectral+C2R+DWT) and one step launch */
    int timed_chunks;           /* number of chunks those means average over */
    int first_primal_below;     /* first k with primal(y^(k)) <= target_objective (0: none) */
    wdb_status status;
    /* params.kkt_check = 1 (else NaN): FP64 check of the returned x, as wdb_theta_kkt */
    double kkt_off, kkt_on;     /* KKT residuals of x (see wdb_kkt_result) */
    double gap64, rel_gap64;    /* duality gap of x from FP64 r and g, and gap / E(x) */
} wdb_solve_result;

/* FP64 optimality check of an iterate (wdb_theta_kkt). */
typedef struct {
    double objective;           /* E(x) = 1/2 ||Theta_K x - x0||^2 + sum w|x| */
    double gap, rel_gap;        /* E(x) - D(-s r), s = min(1, 1/max_i |g_i|/w_i); gap / E(x) */
    double kkt_off;             /* max over all i of (|g_i| - w_i)_+ / w_i */
    double kkt_on;              /* max over x_i != 0 of |g_i + w_i sign(x_i)| / w_i */
    double gmax;                /* max_i |g_i| / w_i */
    long long support;          /* nonzero coefficients of x */
} wdb_kkt_result;

/* ---- Theta_K construction (Algorithm 2 + Sec. 3.7), FP64 on the device ----
 * For every subband b (3J+1 of them) the wavelet at position 0 is blurred with H and H^T
 * (cuFFT, FP64) and analysed by one forward DWT (the column and row probes of Algorithm 2).
 * Blocks whose output subband is finer than or as fine as the input take column taps, the
 * others row taps (Thm 3). Whole taps are kept in the order of decreasing score |sigma_b v|
 * (sigma_b = 2^{s_b} for WDB_RULE_WEIGHTED, 1 for WDB_RULE_NAIVE; ties by (a, b, oy, ox)
 * ascending) while the entry count stays <= K; |v| <= 1e-14 max|v| is never kept.
 * K >= N^2 keeps every tap. The diagonals of Theta_K^T Theta_K and of its square are
 * computed per phase class for the preconditioners (Sec. 4.2, 4.3).
 * Returns WDB_EINVAL for sizes not divisible by 2^levels, an even or larger-than-image
 * PSF, K < 0, an unknown wavelet, or levels < 1. On success *out owns device memory
 * until wdb_theta_free. The call synchronises `stream`. */
wdb_status wdb_build_theta(const double* psf_host, int kh, int kw, int n_rows, int n_cols,
                           const char* wavelet, int levels, long long K, int rule,
                           void* stream, wdb_theta** out);

/* Build a handle from an explicit tap list (host arrays of length n_taps). Tap t gives the
 * value v[t] to the circulant diagonal (oy[t], ox[t]) of block (a[t], b[t]) in the
 * convention of Algorithm 2: if level(a) <= level(b) the entry ((a,p),(b,q)) is v when
 * p = (oy,ox) + 2^{level(b)-level(a)} q (mod the sides of a); otherwise when
 * q = (oy,ox) + 2^{level(a)-level(b)} p (mod the sides of b). Used to load an operator
 * built elsewhere (e.g. from a file). Duplicate taps are WDB_EINVAL. */
wdb_status wdb_theta_from_taps(int n_rows, int n_cols, const char* wavelet, int levels,
                               long long n_taps, const int* a_host, const int* b_host,
                               const int* oy_host, const int* ox_host, const double* v_host,
                               void* stream, wdb_theta** out);

wdb_status wdb_theta_info_get(const wdb_theta* th, wdb_theta_info* info);

/* Copy the kept taps to host arrays (capacity cap >= info.n_taps), sorted by (a, b, oy, ox). */
wdb_status wdb_theta_export_taps(const wdb_theta* th, long long cap, int* a_host, int* b_host,
                                 int* oy_host, int* ox_host, double* v_host);

/* Preconditioner table and step for `precond` (computed on first use and cached):
 * P_host receives 4^J FP64 values, one per phase class (subband b, qy mod R_b, qx mod R_b),
 * R_b = 2^{J - level(b)}, subbands in planar order, phases row-major; tau and L_hat are the
 * step 1/(1.01 L_hat) and the power-iteration estimate of lambda_max(P^-1/2 M P^-1/2)
 * (Algorithm 3, step size). Md_host / M2d_host (optional, 4^J each) receive diag(M) and
 * diag(M^2). Any output pointer may be NULL. Synchronises `stream`. */
wdb_status wdb_theta_precond(wdb_theta* th, int precond, double jacobi_eps, void* stream,
                             double* P_host, double* Md_host, double* M2d_host,
                             double* tau_host, double* L_hat_host);

/* Override the preconditioner table (4^J values, > 0) and step used for `precond`. */
wdb_status wdb_theta_set_precond(wdb_theta* th, int precond, const double* P_host, double tau);

/* Replace the plans of the FP32 Theta_K / Theta_K^T kernels (autotuned on the GPU by
 * wdb_build_theta and wdb_theta_from_taps) by the planner's plans for a staging buffer of
 * smem_budget bytes (<= 0: 32768; at most 98304), tiles whose modelled cost stays under
 * cap_share CTA shares (<= 0: 2), and either tiles above split_share CTA shares split at
 * batch boundaries over several CTAs (<= 0: none), whose partial sums the last part to
 * finish adds in part order, or (super_tiles = 1) work items of 2 x 2 tiles of side 32
 * staged together wherever all their regions fit one buffer, or (super_tiles = 2) grouped
 * items: one item computes the tile of every subband of a level (A_J with the level-J
 * details), staging each input region once for all of them. Results change only by the
 * FP32 summation order. Captured solve graphs of the handle are dropped; the replaced plans'
 * device memory is released with the handle. WDB_EINVAL for a NULL handle, smem_budget >
 * 98304, super_tiles outside 0..2, or split_share > 0 together with super_tiles.
 * Synchronises `stream`. */
wdb_status wdb_theta_replan(wdb_theta* th, int smem_budget, double cap_share, double split_share, int super_tiles,
                            void* stream);

/* Planner self-check on the host (no GPU needed). Builds the tile plan of Theta_K
 * (transpose = 0) or Theta_K^T (1) for a tap list in the convention of wdb_theta_from_taps,
 * for element size esize (4: FP32, 8: FP64), a staging buffer of smem_budget bytes (<= 0:
 * 32768), cap_share, split_share and super_tiles as in wdb_theta_replan, balanced for `ctas`
 * CTAs (<= 0: 456), and checks its structural invariants: every output of every subband
 * produced exactly once, every staged region and tap area inside the staging buffer, every
 * staged read inside its pair's region, and the conditions of super tiles, split tiles and
 * 16-byte staging. Fills *summary (may be NULL). WDB_EPLAN: an invariant is broken
 * (wdb_last_error names the first); WDB_EINVAL: bad sizes, subband indices or esize. */
typedef struct {
    int items, pairs, batches, split_tiles, super_subbands, smem_bytes;
    long long macs;             /* multiply-adds of one application (padding included) */
    int groups;                 /* groups of subbands worked together (super_tiles = 2) */
} wdb_plan_summary;
wdb_status wdb_tile_plan_check(int n_rows, int n_cols, int levels, long long n_taps, const int* a_host,
                               const int* b_host, const int* oy_host, const int* ox_host, const double* v_host,
                               int transpose, int esize, int smem_budget, double cap_share, double split_share,
                               int super_tiles, int ctas, wdb_plan_summary* summary);

/* Serialise / restore a handle (taps, layout, wavelet; preconditioners are recomputed). */
wdb_status wdb_theta_save(const wdb_theta* th, const char* path);
wdb_status wdb_theta_load(const char* path, void* stream, wdb_theta** out);
void wdb_theta_free(wdb_theta* th);

/* One operator application (Eq. gradientapprox pieces): out = Theta_K in (transpose = 0) or
 * Theta_K^T in (transpose = 1); N floats each, device. */
wdb_status wdb_theta_apply(const wdb_theta* th, const float* in_dev, float* out_dev,
                           int transpose, void* stream);

/* ---- Solvers ----
 * wdb_solve: Algorithm 3 on Theta_K. x0 = Psi* u0 is computed on the device (FP32), then
 * for k = 1, 2, ...: r = Theta_K y - x0 (kernel 1), g = Theta_K^T r fused with
 * x = soft(y - tau g / P, tau w / P) and y = x + (k-1)/(k+2)(x - x_prev) (kernel 2).
 * Iterates are FP32; the objective and duality-gap reductions are FP64 above the warp level.
 * u_dev: N floats (image); x_dev: N floats (coefficients, output). Synchronises `stream`.
 * result->status repeats the return value. */
wdb_status wdb_solve(wdb_theta* th, const float* u_dev, float* x_dev,
                     const wdb_solve_params* params, void* stream, wdb_solve_result* result);

/* Same with the data already in the wavelet domain: x0_dev = Psi* u0 (N floats). */
wdb_status wdb_solve_coeffs(wdb_theta* th, const float* x0_dev, float* x_dev,
                            const wdb_solve_params* params, void* stream,
                            wdb_solve_result* result);

/* Batched solve (many problems of uneven size, each with its own Theta_K handle, image,
 * weights and stopping rule): the problems advance together, two launches per iteration
 * that cover the tiles of every running problem, heaviest first, in chunks of check_every
 * iterations replayed as a CUDA graph; a problem that meets its own stopping rule drops out.
 * th[b], u_dev[b], x_dev[b], params[b], results[b] for b < B; every handle distinct; all
 * problems share check_every. results[b].objective is the exact FP64 objective of x_dev[b];
 * results[b].support is -1 (not counted); solve_ms is the wall time of the whole call.
 * Synchronises `stream`. */
wdb_status wdb_solve_batch(int B, wdb_theta* const* th, const float* const* u_dev, float* const* x_dev,
                           const wdb_solve_params* params, void* stream, wdb_solve_result* results);

/* Objective E(x) = 1/2||Theta_K x - x0||^2 + sum w|x| in FP64 for device x, x0. */
wdb_status wdb_theta_objective(const wdb_theta* th, const float* x_dev, const float* x0_dev,
                               double lambda, const double* w_subband_host, void* stream,
                               double* E_host);

/* FP64 check of the first-order optimality conditions of the l1 problem at a device iterate x
 * (the conditions whose identification Sec. 4 discusses: |g_i| <= w_i everywhere and
 * g_i = -w_i sign(x_i) on the support, g = Theta_K^T (Theta_K x - x0)): r and g are computed
 * with FP64 taps and FP64 accumulation on the device from the FP32 x and x0 (N floats each),
 * the residuals, objective and duality gap reduced in FP64. Residuals are relative to w_i
 * (absolute where w_i = 0). Allocates 16 N bytes of FP64 workspace in the handle on first use.
 * WDB_EINVAL for NULL arguments. Synchronises `stream`. */
wdb_status wdb_theta_kkt(wdb_theta* th, const float* x_dev, const float* x0_dev, double lambda,
                         const double* w_subband_host, void* stream, wdb_kkt_result* out);

/* Exact operator A = H Psi for the FFT path (Algorithm 1 gradient, Sec. 5.2): cuFFT FP32
 * R2C/C2R for the solve, FP64 for the preconditioner diagonals (constant per subband, the
 * full Theta having full translation symmetry) and the power iteration. */
wdb_status wdb_fftop_create(const double* psf_host, int kh, int kw, int n_rows, int n_cols,
                            const char* wavelet, int levels, void* stream, wdb_fftop** out);
void wdb_fftop_free(wdb_fftop* op);
wdb_status wdb_fftop_precond(wdb_fftop* op, int precond, double jacobi_eps, void* stream,
                             double* P_host /* 3J+1 */, double* tau_host, double* L_hat_host);
wdb_status wdb_fftop_set_precond(wdb_fftop* op, int precond, const double* P_host, double tau);

/* Exact objective 1/2||H Psi x - u0||^2 + sum w|x| of a device iterate x (N floats) for the
 * device image u0 (the FP32 spectral path of wdb_solve_fft, FP64 reductions), e.g. to measure
 * a Theta_K solution on the exact problem. Synchronises `stream`. */
wdb_status wdb_fftop_objective(wdb_fftop* op, const float* u_dev, const float* x_dev, double lambda,
                               const double* w_subband_host, void* stream, double* E_host);

/* FISTA with the exact gradient: per iteration IDWT(y), R2C, r^ = h^ z^ - u0^ with
 * Parseval reductions, g^ = conj(h^) r^, C2R, DWT, then the same fused step as wdb_solve.
 * result->objective is the exact objective 1/2||H Psi x - u0||^2 + sum w|x|. */
wdb_status wdb_solve_fft(wdb_fftop* op, const float* u_dev, float* x_dev,
                         const wdb_solve_params* params, void* stream, wdb_solve_result* result);

/* ---- Spatially varying blur (Sec. 3.1, 3.4, 3.5) ----
 * H spreads every input pixel of image row i with its own PSF psfs[i] (odd kh x kw, origin at
 * (kh/2, kw/2)) on the torus: (H u)[(i+a) mod R][(j+b) mod C] += psfs[i][a+kh/2][b+kw/2] u[i][j].
 * (One PSF for every row is the convolution of wdb_build_theta.) Such an H commutes with
 * horizontal translations, so Theta = Psi* H Psi is circulant along the column axis inside
 * every pair of subbands, and a tap is (a, py, b, qy, ox): output row py of subband a, input
 * row qy of subband b, horizontal diagonal ox, with the entries
 *   ((a, py, px), (b, qy, qx)) for px = ox + 2^{level(b)-level(a)} qx (mod C_a) when
 *   level(a) <= level(b) (C_b entries), otherwise qx = ox + 2^{level(a)-level(b)} px
 *   (mod C_b) (C_a entries).
 * Construction (Sec. 3.4, one probe per subband row): H applied to the wavelet of (b, qy, 0)
 * for every input row and H^T to the wavelet of (a, py, 0) for every output row of a subband
 * above level 1, one FP64 forward DWT each, on the device. Thresholding (Sec. 3.7): whole taps
 * by decreasing score |sigma_b v| (sigma_b = 2^{level(b)} or 1 as in wdb_build_theta), ties by
 * (a, py, b, qy, ox) ascending, while the entry count stays <= K; |v| <= 1e-14 max|v| is never
 * kept. Preconditioner classes: (b, qy, qx mod 2^{J - level(b)}), one table entry per class,
 * subbands in planar order, then row-major in (qy, qx mod 2^{J - level(b)}) (info.n_classes).
 * Limits: n_cols <= 2048 (WDB_EUNSUPPORTED above), n_rows, n_cols divisible by 2^levels,
 * kh <= n_rows, kw <= n_cols. The build holds one FP64 candidate per coefficient window of
 * every probe on the device (info.candidate_slots x 8 bytes) while it runs. */
typedef struct {
    int n_rows, n_cols, levels, n_subbands;
    int rule;
    long long K_requested;      /* K passed to wdb_vtheta_build */
    long long K_eff;            /* nonzero entries of Theta_K (<= K_requested) */
    long long n_taps;           /* kept taps */
    long long n_candidates;     /* nonzero taps of the full Theta (0 for wdb_vtheta_from_taps) */
    long long candidate_slots;  /* FP64 candidate values stored by the build */
    int n_probes;               /* probes (column and row) of the build */
    int n_classes;              /* length of the preconditioner tables */
    int n_plan_rows;            /* output rows of one application (CTAs of a launch) */
    long long plan_taps[2];     /* taps of the Theta_K and Theta_K^T row plans */
    double theta_max_abs;       /* max |tap| of the full Theta */
    double build_ms;            /* wall time of the build, device work included */
} wdb_vtheta_info;

/* psfs_host: n_rows x kh x kw FP64, row-major. K >= 0; rule WDB_RULE_*. WDB_EINVAL for bad
 * sizes, an even PSF side, a non-finite PSF value, K < 0 or an unknown wavelet. Synchronises
 * `stream`; on success *out owns device memory until wdb_vtheta_free. */
wdb_status wdb_vtheta_build(const double* psfs_host, int kh, int kw, int n_rows, int n_cols,
                            const char* wavelet, int levels, long long K, int rule, void* stream,
                            wdb_vtheta** out);
/* A handle from an explicit tap list (host arrays, n_taps each) in the convention above.
 * Taps outside the subbands' sides, or a duplicate (a, py, b, qy, ox), are WDB_EINVAL. */
wdb_status wdb_vtheta_from_taps(int n_rows, int n_cols, const char* wavelet, int levels, long long n_taps,
                                const int* a_host, const int* py_host, const int* b_host, const int* qy_host,
                                const int* ox_host, const double* v_host, void* stream, wdb_vtheta** out);
wdb_status wdb_vtheta_info_get(const wdb_vtheta* op, wdb_vtheta_info* info);
/* Kept taps to host arrays (capacity cap >= info.n_taps), sorted by (a, py, b, qy, ox). */
wdb_status wdb_vtheta_export_taps(const wdb_vtheta* op, long long cap, int* a_host, int* py_host, int* b_host,
                                  int* qy_host, int* ox_host, double* v_host);
/* out = Theta_K in (transpose = 0) or Theta_K^T in (1); N floats each, device. */
wdb_status wdb_vtheta_apply(const wdb_vtheta* op, const float* in_dev, float* out_dev, int transpose,
                            void* stream);
/* Preconditioner of kind `precond` (computed on first use, cached): P_host, Md_host, M2d_host
 * receive info.n_classes values each (diag(M), diag(M^2) of M = Theta_K^T Theta_K per class,
 * FP64 on the host from the taps); tau, L_hat as for wdb_theta_precond (FP64 power iteration on
 * the device). Any output may be NULL. Synchronises `stream`. */
wdb_status wdb_vtheta_precond(wdb_vtheta* op, int precond, double jacobi_eps, void* stream, double* P_host,
                              double* Md_host, double* M2d_host, double* tau_host, double* L_hat_host);
/* Override the table (info.n_classes values > 0) and step used for `precond`. */
wdb_status wdb_vtheta_set_precond(wdb_vtheta* op, int precond, const double* P_host, double tau);
/* Algorithm 3 on this Theta_K, as wdb_solve / wdb_solve_coeffs (params.kkt_check is ignored;
 * the kkt_* and *64 result fields are NaN). */
wdb_status wdb_vtheta_solve(wdb_vtheta* op, const float* u_dev, float* x_dev, const wdb_solve_params* params,
                            void* stream, wdb_solve_result* result);
wdb_status wdb_vtheta_solve_coeffs(wdb_vtheta* op, const float* x0_dev, float* x_dev,
                                   const wdb_solve_params* params, void* stream, wdb_solve_result* result);
/* E(x) = 1/2||Theta_K x - x0||^2 + sum w|x| in FP64 for device x, x0. */
wdb_status wdb_vtheta_objective(wdb_vtheta* op, const float* x_dev, const float* x0_dev, double lambda,
                                const double* w_subband_host, void* stream, double* E_host);
void wdb_vtheta_free(wdb_vtheta* op);
/* Host self-check of the row plans (no GPU): builds the plan of Theta_K (transpose = 0) or
 * Theta_K^T (1) for a tap list in the convention above, runs one application on the host with
 * the kernel's index arithmetic, checking every row, tap and access against the vector
 * bounds, and writes y_host = Theta_K x_host (or the transpose) in FP64 (N values each).
 * WDB_EPLAN: an invariant broke (wdb_last_error names it); WDB_EINVAL: bad sizes or taps. */
wdb_status wdb_vtheta_plan_check(int n_rows, int n_cols, const char* wavelet, int levels, long long n_taps,
                                 const int* a_host, const int* py_host, const int* b_host, const int* qy_host,
                                 const int* ox_host, const double* v_host, int transpose, const double* x_host,
                                 double* y_host);

/* ---- Wavelet transforms (Sec. 2), FP32, device ---- */
wdb_status wdb_dwt(const float* img_dev, float* coef_dev, int n_rows, int n_cols,
                   const char* wavelet, int levels, void* stream);
wdb_status wdb_idwt(const float* coef_dev, float* img_dev, int n_rows, int n_cols,
                    const char* wavelet, int levels, void* stream);

/* Forward transform that allocates nothing (the paper has no counterpart; this is a service
 * for callers that cannot allocate device memory: code running inside another framework's
 * locked-down memory pool, real-time paths where cudaMalloc and the synchronisation it may
 * imply are not allowed, or callers holding a capture or lock that an allocation would
 * break). Same result as wdb_dwt, but the intermediate approximations live in a file-scope
 * device array of 4 Mi floats (16 MiB) that a GPU keeps until the process exits once the
 * library's code has been loaded on it; images above 8 Mi - 2 pixels are rejected with
 * WDB_EINVAL. The first call on each device looks the array's device address up, with that
 * device current; under lazy module loading (CUDA_MODULE_LOADING=LAZY, PyTorch's default)
 * that lookup is also what loads the module holding the array, which reserves its 16 MiB
 * and may synchronise the device, so make the first call on every device during set-up,
 * before any stream capture and outside any section that must not allocate. Later calls on
 * that device allocate nothing. The looked-up address is kept for the life of the process:
 * after a cudaDeviceReset of that device the function must not be called on it again. All
 * calls share the array: calls that overlap on the GPU (other streams, other threads) race
 * and must be serialised by the caller. No cudaMalloc, cudaFree or allocating library
 * routine is called. */
wdb_status wdb_dwt_noalloc(const float* img_dev, float* coef_dev, int n_rows, int n_cols,
                           const char* wavelet, int levels, void* stream);

/* Filter taps of a wavelet (host): h (low-pass) and g (high-pass) of length 2p. */
wdb_status wdb_wavelet_filters(const char* wavelet, int cap, double* h_host, double* g_host,
                               int* taps);

/* ---- Learned warm start (an addition to the paper's method) ----
 * A U-Net v = u + N(u) maps a blurred image u to an image whose wavelet coefficients
 * x_init = Psi* v start FISTA (wdb_solve_params.x_init_dev); with a good start Algorithm 3
 * reaches its stopping rule in fewer iterations, and the solver's own stop keeps the result
 * the minimiser of the same problem. Architecture: `levels` resolutions, `channels` (<= 32)
 * feature maps, periodic 3x3 convolutions with bias and ReLU, 2x2 average pooling down,
 * nearest 2x upsampling plus skip addition up; the output convolution is added to u.
 * Storage: BF16 activations and weights, FP32 accumulation, FP32 master weights, gradients
 * and Adam moments. Images are [B][height][width] FP32 in device memory.
 * Parameter vector (FP32, host): per convolution W as [C_out][C_in][3][3] then b, in the
 * order in, e0, e1a, e1b, ..., e(L-1)a, e(L-1)b, d(L-2)a, d(L-2)b, ..., d0a, d0b, out.
 * height and width must be divisible by 2^(levels-1); 1 <= B <= max_batch. */
typedef struct wdb_cnn wdb_cnn;
wdb_status wdb_cnn_create(int levels, int channels, int height, int width, int max_batch,
                          unsigned long long seed, void* stream, wdb_cnn** out);
void wdb_cnn_free(wdb_cnn* net);
long long wdb_cnn_num_params(const wdb_cnn* net);
/* Replace the FP32 parameters (count = wdb_cnn_num_params) and reset the Adam state. */
wdb_status wdb_cnn_set_params(wdb_cnn* net, const float* params_host, long long count, void* stream);
wdb_status wdb_cnn_get_params(const wdb_cnn* net, float* params_host, long long cap);
/* v_dev = network(u_dev), both [B][height][width]. */
wdb_status wdb_cnn_forward(wdb_cnn* net, const float* u_dev, float* v_dev, int B, void* stream);
/* loss = mean((network(u) - target)^2) (FP64 reduction); grad_host (may be NULL) receives
 * the FP32 gradient of every parameter. Synchronises `stream`. */
wdb_status wdb_cnn_loss_grad(wdb_cnn* net, const float* u_dev, const float* target_dev, int B,
                             void* stream, double* loss_host, float* grad_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on that loss. */
wdb_status wdb_cnn_train_step(wdb_cnn* net, const float* u_dev, const float* target_dev, int B,
                              double lr, void* stream, double* loss_host);
/* Checkpoint: shape, step count, seed, parameters and Adam moments. */
wdb_status wdb_cnn_save(const wdb_cnn* net, const char* path);
wdb_status wdb_cnn_load(const char* path, void* stream, wdb_cnn** out);
/* wdb_solve started from the network: x_init = Psi* network(u) when its objective E is below
 * that of x = 0 (E(0) = 1/2 ||Psi* u||^2), else the cold start x = 0 (the fallback);
 * *start_used (may be NULL) reports 1 (network) or 0 (cold). The network must have the
 * operator's image size and params->x_init_dev must be NULL. The stopping rule is the
 * caller's, so the result solves the same problem as wdb_solve. Synchronises `stream`. */
wdb_status wdb_solve_warm(wdb_theta* th, wdb_cnn* net, const float* u_dev, float* x_dev,
                          const wdb_solve_params* params, void* stream, wdb_solve_result* result,
                          int* start_used);

/* ---- Diagnostics ---- */
const char* wdb_status_str(wdb_status s);
const char* wdb_last_error(void);
/* Number of kernels this library launched (or placed in graphs that were launched) since
 * load or the last reset; counts graph replays node by node. */
long long wdb_kernel_launches(int reset);

#ifdef __cplusplus
}
#endif
#endif /* WDB_H */
