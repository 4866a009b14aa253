"""Plain FP64 CPU oracle for the phaseless-AFQMC walker step (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import, call or execute anything in
this package.  The product path (the CUDA library under ``paper_2209_04015_b300``
and its Python binding) never imports it, and the two share no code: no kernels,
headers, helpers, constants or pre/post-processing.  Inputs reach both sides from
``paper_2209_04015_b300.synthetic``, which holds no arithmetic of the method.

Modules
-------
afqmc     one imaginary-time step, local energy and QR re-orthogonalisation,
          written step by step from the paper (arXiv:2209.04015) in float64 /
          complex128 NumPy.
philox    Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the
          Box-Muller map to Gaussian auxiliary fields.
gradients closed-form gradients of the mixed local energy.
chain     the objective of a K-step chain (fixed fields, detached weights) through
          the NumPy oracle, and the same steps in PyTorch CPU float64 whose
          autograd gives the chain's gradient.

Every function says which passage of the paper it follows.  Where the paper is
silent or ambiguous the reading taken is stated in the function's docstring.
"""
