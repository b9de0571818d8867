"""ORACLE -- test infrastructure only.

A plain FP64 CPU implementation of the muffin-tin H and S of the FLAPW method,
written from the paper's definitions (App. A, Eqs. def_overlap, def_hamilton)
and used to check the CUDA library. Only tests/, the smoke check and the
benchmark's CPU-baseline leg may import it. It shares no code with the CUDA
library and never imports it.
"""
from .hsref import (  # noqa: F401
    load,
    sbessel,
    ylm,
    wigner3j,
    gaunt,
    T_matrix,
    cholesky,
    T_hpd_info,
    coefficients,
    build_HS,
    HS_entries,
    HS_columns,
    HS_brute,
    threads,
)
from .reduce import hermitian_from_triangle, reduce_generalized  # noqa: F401
