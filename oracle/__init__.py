"""FP64 CPU oracle for wavelet-domain l1-l2 deblurring (Escande & Weiss, arXiv 1512.08401).

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously correct restatement
of the paper's method in numpy/scipy float64, written so that a reader can check it
against the paper by eye. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it. The CUDA library never calls it and shares no code,
tables or constant generators with it.

Modules
-------
wavelet   Daubechies filters (spectral factorisation) and the periodic separable DWT (Sec. 2).
blur      Direct periodic convolution H and its adjoint (Sec. 3.6, translation operator).
theta     Theta = Psi* H Psi: dense brute force (Eq. matrixH), probe construction
          (Algorithm 2), circulant block expansion (Def. rectangular circulant, Thm 3),
          naive / weighted K-sparse thresholding (Sec. 3.7).
precond   Jacobi and SPAI diagonal preconditioners (Sec. 4.2, 4.3), power iteration for
          the Lipschitz constant in the P-metric (Algorithm 3 step size).
solver    Preconditioned FISTA (Algorithm 3) on Theta_K, exact-operator FISTA
          (Algorithm 1 with the FFT-path gradient evaluated by direct convolution),
          objective, duality gap, KKT residuals, and a coordinate-descent Lasso solver
          used only to pin FISTA.
varying   Row-varying blur (Sec. 3.1, 3.5): H by direct scatter, Theta from one probe per
          subband row with horizontal circulant taps (Sec. 3.4), tap thresholding (Sec. 3.7)
          and the preconditioner classes of that operator.
rng       splitmix64 counter-based generator (Steele, Lea & Flood 2014) for the power
          iteration start vector.
cnn       FP64 forward/backward of the warm-start U-Net (not a paper component).

Every function says which passage of the paper it follows. Functions whose results are not
pinned by a test against something other than themselves say "parity unpinned".
"""
