"""FP64 CPU oracle for the CoNet-Rx hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes anything under ``oracle/``; only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference arm may use it.  The oracle is a
plain, slow, obviously correct restatement of what the paper's receiver computes:

* ``philox``   counter-based RNG (Salmon et al., SC'11) driving every random draw
* ``sim``      the OFDM link of Sec. II, Eq. (1): bits, Gray QAM, fixed pilots,
               TDL Rayleigh channel with Doppler, interferer, AWGN
* ``rx``       input assembly (Sec. II-A), LS, LS-LMMSE receiver (Sec. I, Sec. IV
               baselines), exact / max-log demapping, bit-error counting
* ``net``      CoNet forward and backward (Sec. III, Fig. "Example I", RB, MRB),
               BCE loss and Adam

Everything is float64 numpy; library routines (matmul, einsum) serve only as the
steps their definitions name.  Functions whose result has no independent pin say
"parity unpinned" in their docstring.
"""
