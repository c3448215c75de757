"""CPU oracle for the Toeplitz OLS / AR(p) problem — test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg may import it. The CUDA
library never imports it and shares no code with it.
"""
from .tols import (LsarResult, OracleSolution, RHResult, compressed_ols, exact_leverage, generalized_leverage,
                   gram, hadamard_transform, lag_matrix, leverage_p1, leverage_sample, leverage_step, lsar, matvec,
                   ols_qr, pacf, repeated_halving, residual_check, rh_lsar, rmatvec, row_norms, srht_ols)
