"""FP64 CPU oracle for decentralized feedforward L-MMSE equalization.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path and never imports it; the product path never calls it.

Modules
-------
``lmmse``   PD and FD L-MMSE equalization, error variances and optimal fusion
            (Sec. II-B..D, Sec. III-A, Sec. IV-A, Lemma 1, Thm. 3).
``linear``  PD and FD with the MRC and ZF equalizers of Sec. III-A in place of
            L-MMSE (FD fuses them with the same optimal weights).
``lama``    LAMA-PD (Algorithm 1 on the PD pair) and LAMA-FD (per cluster, then
            the optimal fusion), with the posterior-mean denoiser of Eq. F.
``llr``     max-log soft outputs for square QAM (the paper names LLRs but gives
            no formula; the reading is stated in that module).
``adjoint`` the differentiable FD form (per-cluster regularizers, free fusion
            weights) and its closed-form gradients, checked by finite differences.
``theory``  large-system closed forms and fixed points (Thm. 1, Cor. 1,
            Lemma 2, Lemma 4, Lemma 5, Lemma 7) and the Sec. VI message sizes.

Every function works in float64/complex128 on the complex64 inputs it is
given (they are upcast once), loops over subcarriers in plain Python and uses
library primitives (``numpy.linalg.inv``, matrix products) only as steps of the
paper's definitions, so it can be checked against the paper by eye.
"""
from . import adjoint, lama, linear, llr, lmmse, theory  # noqa: F401
