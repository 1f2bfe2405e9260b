"""FP64 CPU oracle for the SHGEMM random projection, randomized SVD and RP-HOSVD.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
``libshg.so`` and its Python binding ``paper_2304_04612_gb300``) imports,
links or executes anything in this package.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm
may call it.

Everything here is a plain, slow, obviously-correct restatement of the paper
(Ootomo & Yokota, "Mixed-Precision Random Projection for RandNLA on Tensor
Cores", arXiv 2304.04612) in float64 with numpy.  Library primitives (matmul,
Householder QR, SVD) serve as single steps; there is no blocking, fusion or
reordering beyond what the paper's definitions state.

Modules
-------
``lowp``     eXmY rounding (RN, ties-to-even) and decoding         (Sec. 3.1, Eq. g-fp-error)
``gaussian`` Table 1 quantities, alpha_Y, Philox4x32-10 + Box-Muller (Sec. 3.2, Table 1)
``shgemm``   exact product, SHGEMM split emulation, error bounds     (Sec. 4.1-4.4)
``rsvd``     randomized SVD with optional power scheme               (Algorithm 1, Sec. 2.1-2.2)
``hosvd``    random-projection HOSVD                                  (Algorithm 2, Sec. 5.2)
``sketch``   learned-sketch loss and its closed-form gradient         (Theorems 1 and 3 for the estimator)

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, a printed value of the paper, a library special case or brute
force, except where its docstring says "parity unpinned".
"""
