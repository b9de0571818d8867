"""Operation counts and memory figures (host-side bookkeeping).

Two conventions are kept side by side:

* ``algorithmic_flops`` -- what this library's path must compute for one
  k-point: the upper triangle (diagonal included) of H = W^H X and
  S = W^H Y with depth D = 2 sum_a N_La (8 real flops per complex
  multiply-add), plus the T-apply X_a = T_a W_a (8 flops per complex
  multiply-add, full 2N_La x 2N_La blocks). This is the numerator of every
  effective TFLOP/s figure.
* ``paper_listing_flops`` -- the counts printed next to the paper's BLAS
  listings (Sec. 4.3-4.6), with the HPD fraction of the T^[AA] matrices as a
  parameter; and ``paper_memory_bytes``, the footprint formula of Sec. 4.8.
"""
from __future__ import annotations

from typing import Iterable


def algorithmic_flops(n_g: int, nl_per_atom: Iterable[int]) -> dict:
    nls = list(nl_per_atom)
    depth = 2 * sum(nls)
    tri = n_g * (n_g + 1) // 2
    f_hs = 2 * 8 * tri * depth  # H and S, triangle only
    f_t = 8 * n_g * sum((2 * n) ** 2 for n in nls)  # X_a = T_a W_a
    return {"F_HS": float(f_hs), "F_T": float(f_t), "total": float(f_hs + f_t), "depth": depth}


def paper_listing_flops(n_a: int, n_l: int, n_g: int, hpd_fraction: float = 0.5) -> dict:
    """Counts of Listings alg:S, alg:H_BB and alg:H_AA (dynamic HPD routing)."""
    na, nl, ng, h = float(n_a), float(n_l), float(n_g), float(hpd_fraction)
    s_big = 8 * na * nl * ng ** 2                      # two zherk
    s_small = 2 * na * nl * ng                         # row scaling by U
    hbb_big = 8 * na * nl * ng ** 2                    # zher2k
    hbb_small = 16 * na * nl ** 2 * ng                 # zgemm + zhemm per atom
    haa_big = (1 - h) * 8 * na * nl * ng ** 2 + h * 4 * na * nl * ng ** 2  # zgemm / zherk
    haa_small = h * na * (4.0 / 3.0 * nl ** 3 + 4 * nl ** 2 * ng) + (1 - h) * na * 8 * nl ** 2 * ng
    big = s_big + hbb_big + haa_big
    small = s_small + hbb_small + haa_small
    return {"big": big, "small": small, "share": big / (big + small)}


def paper_memory_bytes(n_a: int, n_l: int, n_g: int, backup: bool = True) -> float:
    """Footprint of the paper's final algorithm (Sec. 4.8)."""
    ab = 32.0 * n_a * n_l * n_g
    hs = 32.0 * n_g ** 2
    return ab + hs + (max(ab - 16.0 * n_g ** 2, 0.0) if backup else 0.0)
