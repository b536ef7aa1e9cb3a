"""FP64 CPU oracle for block-splitting ADMM over random Fourier features.

This package is TEST INFRASTRUCTURE. It exists to check the GPU library, not to
be one: only the test suite, the smoke check in ``__graft_entry__`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The
product path (the CUDA library and its Python binding) never imports, links or
executes anything here, and this package never imports the product.

Everything is plain numpy in float64, written to be read against the paper
(Sindhwani & Avron, "High-performance Kernel Machines with Implicit Distributed
Optimization and Randomization", arXiv:1409.0940):

* ``philox``  -- Philox4x32-10 counter-based generator (Salmon et al., SC'11) and
                 the random Fourier feature parameters drawn from it (Sec. 4).
* ``rff``     -- the explicit feature matrix Z = sqrt(2/D) cos(X G + b) (Sec. 4),
                 block partitions (Sec. 3), the Gaussian kernel (Sec. 4).
* ``prox``    -- proximal operators of the losses and regularisers (Sec. 2.3,
                 Sec. 3 "Modularity").
* ``admm``    -- block-splitting ADMM in its equation form (Sec. 3, the update
                 equations around eq. (gp), (obar_ij), (obar)), the memory-
                 efficient reorganisation (Sec. 3, the U_ij / Delta rewrite),
                 graph projection (eq. (graphU), (graphV)), the ridge closed form
                 (Sec. 2.2), residuals, objective and prediction.
* ``memory``  -- the per-node memory model, eq. (mem).
* ``fastfood`` -- Fastfood's structured projection (Sec. 4 lists the map).
* ``tensorsketch`` -- TensorSketch features of the polynomial kernel, one independent
                 sketch per column block (Sec. 4 lists the map and the block assembly).

Parity status of every function is stated in its module header; all functions
here are pinned by the CPU tests (closed forms, brute force, published known-
answer vectors, identities the paper states), none is "parity unpinned".
"""
