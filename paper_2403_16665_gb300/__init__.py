"""GB300-native alpha-densified DFT (arxiv 2403.16665), CUDA kernels behind a C ABI.

    from paper_2403_16665_gb300 import alpha_dft
    X = alpha_dft(x_cuda, alpha=8)      # X[b, m] = (1/N) sum_n x[b, n] exp(-2 pi i m n/(alpha N))
"""
from .autograd import AlphaDFT, alpha_dft_autograd  # noqa: F401
from .adfft import (ALGO_AUTO, ALGO_BLUESTEIN, ALGO_FOLD, ALGO_FOUR_STEP, C64, C128,  # noqa: F401
                    PREC_BF16X3, PREC_FP16X2, PREC_NATIVE, R32, R64, AdfftError, Plan, RaggedPlan,
                    alpha_dft, autotune_clear, autotune_load, autotune_save, load)
