"""CPU FP64 oracle for the von Neumann entropy hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The product path (the CUDA library and its Python
binding) never calls it; it shares no code with the CUDA path, only the
seeded graph inputs of ``paper_2212_09642_gb300.graphs``.

Everything here is plain NumPy / SciPy in float64, written to be read against
Benzi, Rinelli, Simunec (arXiv 2212.09642):

* ``density``    -- rho = L / tr(L) from a graph (Section 2, eq. graph_laplacian)
* ``entropy``    -- S = -sum lambda log lambda by dense eigendecomposition
                    (eq. entropy_definition_eigenvalues) and closed-form
                    Laplacian spectra used to pin it
* ``rng``        -- the counter-based Rademacher generator (SplitMix64 mixer)
* ``krylov``     -- Lanczos quadrature psi_m = ||b||^2 e1^T f(A_m) e1
                    (Section 4, eq. rational-krylov-approximation-quadform)
* ``estimators`` -- Hutchinson, Hutch++ and probing (Section 3)
* ``coloring``   -- greedy distance-d colouring (Algorithm 1)
* ``rational``   -- rational Krylov quadrature with negative real poles
* ``bounds``     -- a-priori (Theorem 2.2, Corollary 3.2, Proposition 4.2)
                    and a-posteriori (Theorem 4.4) error bounds, probing
                    heuristic (Section 5.1)
"""
