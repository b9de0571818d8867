"""Seeded synthetic FLAPW muffin-tin workloads.

The paper's own systems (NaCl, TiO2 taken from FLEUR) are not available, so
these generators stand in for them with the paper's shape relations: N_G about
50-80 plane waves per atom, l_max <= 10, N_L = (l_max+1)^2 <= 121 (Sec. 2.3),
several atoms per species sharing radial data and told apart by a rotation
R_a (App. A.1).

Every array is drawn from numpy's PCG64 with the seed 1602065890 + index, in a
fixed order, so the oracle and the CUDA path always see identical inputs.

What is drawn (per species, per l <= l_max):
  * boundary values u, u', u_dot, u_dot' ~ U[0.2, 1.5], redrawn until the
    Wronskian |u_dot u' - u u_dot'| >= 0.1 (App. A.1 divides by it);
  * ||u_dot_l||^2 ~ U[0.01, 0.5] (Eq. def_overlap);
  * E_l ~ U[-1, 1] (spherical diagonal of Eq. t_matrices);
  * radial integrals I^{(x,y)}_{l,l',l''} ~ U[-1,1] * exp(-l''/2),
    l'' <= 2 l_max (Eq. nonsph_integrals), with the symmetries that follow
    from their definition: I^{(u,u)} and I^{(u_dot,u_dot)} symmetric in
    (l, l'), and I^{(u_dot,u)}_{l,l',l''} = I^{(u,u_dot)}_{l',l,l''}.
Atoms sit at random non-overlapping positions (minimum-image distance
>= R_i + R_j + 0.1) and carry uniformly random proper rotations (Shoemake
quaternions). The plane-wave list K_t = k + G_t takes the N_G vectors of
smallest |K_t|, ties broken by the integer triple of G (Sec. 2.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np

SEED_BASE = 1602065890

CONFIG_NAMES = {
    0: "1 atom, l_max 4, N_G 200, cubic a=8",
    1: "16 atoms / 2 species, l_max 8, N_G 3000",
    2: "64 atoms / 4 species, l_max 10, N_G 12000",
    3: "48 k-points, 32 atoms / 3 species, l_max 6/8/10, N_G 2500-4200",
    4: "256 atoms / 4 species, l_max 10, N_G 20000",
}


@dataclass
class AtomType:
    """Radial data of one species (App. A.1 / A.2)."""

    lmax: int
    rmt: float
    u: np.ndarray
    du: np.ndarray
    udot: np.ndarray
    dudot: np.ndarray
    udot_norm2: np.ndarray
    e_l: np.ndarray
    I_uu: np.ndarray
    I_uud: np.ndarray
    I_udu: np.ndarray
    I_udud: np.ndarray
    T_override: Optional[np.ndarray] = None  # complex (2N_L, 2N_L) or None
    # l_nonsph: the non-spherical (Gaunt) part of T is dense for l, l' <= it;
    # None means l_max (Sec. 3.1, Fig. Tmat_structure)
    lmax_nonsph: Optional[int] = None
    # W_l given by the caller ((l_max+1,) floats), or None: computed from the
    # boundary values as u_dot u' - u u_dot' (App. A.1)
    wronskian: Optional[np.ndarray] = None

    @property
    def nl(self) -> int:
        return (self.lmax + 1) ** 2


@dataclass
class System:
    lattice: np.ndarray  # (3,3) rows a1, a2, a3 (bohr)
    omega: float
    types: List[AtomType]
    type_of_atom: np.ndarray  # (N_A,) int32
    pos: np.ndarray  # (N_A, 3) Cartesian
    rot: np.ndarray  # (N_A, 3, 3) proper rotations

    @property
    def n_atoms(self) -> int:
        return int(self.type_of_atom.shape[0])

    @property
    def sum_nl(self) -> int:
        return int(sum(self.types[int(t)].nl for t in self.type_of_atom))

    def sum_nl2(self) -> int:
        return int(sum(self.types[int(t)].nl ** 2 for t in self.type_of_atom))


@dataclass
class Workload:
    name: str
    system: System
    kvecs: List[np.ndarray] = field(default_factory=list)  # each (N_G, 3)

    @property
    def n_g(self) -> List[int]:
        return [int(k.shape[0]) for k in self.kvecs]


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b1, b2, b3 with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def kpoint_list(lattice: np.ndarray, k_reduced: Sequence[float], n_g: int) -> np.ndarray:
    """The n_g vectors K = k + G of smallest |K| (ties: lexicographic (n1,n2,n3))."""
    lat = np.asarray(lattice, dtype=np.float64)
    b = reciprocal(lat)
    omega = abs(np.linalg.det(lat))
    k = np.asarray(k_reduced, dtype=np.float64) @ b
    kcut = (3.0 * n_g * (2.0 * np.pi) ** 3 / (4.0 * np.pi * omega)) ** (1.0 / 3.0)
    scale = 1.25
    while True:
        kc = kcut * scale + np.linalg.norm(k)
        nmax = [int(np.ceil(kc * np.linalg.norm(lat[i]) / (2 * np.pi))) + 1 for i in range(3)]
        r = [np.arange(-m, m + 1) for m in nmax]
        n1, n2, n3 = np.meshgrid(r[0], r[1], r[2], indexing="ij")
        n = np.stack([n1.ravel(), n2.ravel(), n3.ravel()], axis=1)
        K = k + n @ b
        kn = np.sqrt(np.sum(K * K, axis=1))
        inside = kn <= kcut * scale
        if inside.sum() >= n_g:
            n, K, kn = n[inside], K[inside], kn[inside]
            order = np.lexsort((n[:, 2], n[:, 1], n[:, 0], kn))
            return np.ascontiguousarray(K[order[:n_g]])
        scale *= 1.3


def _draw_type(rng: np.random.Generator, lmax: int, rmt: float) -> AtomType:
    nl1 = lmax + 1
    u = np.empty(nl1)
    du = np.empty(nl1)
    ud = np.empty(nl1)
    dud = np.empty(nl1)
    for l in range(nl1):
        while True:
            a, b, c, d = rng.uniform(0.2, 1.5, size=4)
            if abs(c * b - a * d) >= 0.1:
                break
        u[l], du[l], ud[l], dud[l] = a, b, c, d
    udot_norm2 = rng.uniform(0.01, 0.5, size=nl1)
    e_l = rng.uniform(-1.0, 1.0, size=nl1)
    decay = np.exp(-0.5 * np.arange(2 * lmax + 1))[None, None, :]

    def sym(x):
        iu = np.triu_indices(nl1)
        out = np.empty_like(x)
        for l2 in range(x.shape[2]):
            m = np.zeros((nl1, nl1))
            m[iu] = x[:, :, l2][iu]
            out[:, :, l2] = m + np.triu(m, 1).T
        return out

    I_uu = sym(rng.uniform(-1, 1, size=(nl1, nl1, 2 * lmax + 1)) * decay)
    I_udud = sym(rng.uniform(-1, 1, size=(nl1, nl1, 2 * lmax + 1)) * decay)
    I_uud = rng.uniform(-1, 1, size=(nl1, nl1, 2 * lmax + 1)) * decay
    I_udu = np.ascontiguousarray(np.transpose(I_uud, (1, 0, 2)))
    return AtomType(lmax, rmt, u, du, ud, dud, udot_norm2, e_l,
                    np.ascontiguousarray(I_uu), np.ascontiguousarray(I_uud),
                    I_udu, np.ascontiguousarray(I_udud))


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    u1, u2, u3 = rng.uniform(0.0, 1.0, size=(3, n))
    q0 = np.sqrt(1 - u1) * np.sin(2 * np.pi * u2)
    q1 = np.sqrt(1 - u1) * np.cos(2 * np.pi * u2)
    q2 = np.sqrt(u1) * np.sin(2 * np.pi * u3)
    q3 = np.sqrt(u1) * np.cos(2 * np.pi * u3)
    w, x, y, z = q3, q0, q1, q2
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _random_positions(rng: np.random.Generator, lattice: np.ndarray, radii: np.ndarray) -> np.ndarray:
    lat = np.asarray(lattice, dtype=np.float64)
    inv = np.linalg.inv(lat)
    placed = np.zeros((0, 3))
    placed_r = np.zeros(0)
    for r in radii:
        for _ in range(2000):
            cand = rng.uniform(0.0, 1.0, size=(256, 3)) @ lat
            if placed.shape[0] == 0:
                pick = cand[0]
                break
            d = cand[:, None, :] - placed[None, :, :]
            f = d @ inv
            f -= np.round(f)
            dist = np.sqrt(np.sum((f @ lat) ** 2, axis=2))
            ok = np.all(dist >= placed_r[None, :] + r + 0.1, axis=1)
            if ok.any():
                pick = cand[int(np.argmax(ok))]
                break
        else:
            raise RuntimeError("could not place non-overlapping muffin tins")
        placed = np.vstack([placed, pick[None, :]])
        placed_r = np.append(placed_r, r)
    return placed


def make_system(seed: int, lattice, species: Sequence[tuple], counts: Sequence[int],
                at_origin: bool = False, identity_rot: bool = False) -> System:
    """species: [(lmax, rmt), ...]; counts: atoms per species (atoms grouped by species)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lat = np.asarray(lattice, dtype=np.float64)
    types = [_draw_type(rng, lm, r) for (lm, r) in species]
    toa = np.concatenate([np.full(c, i, dtype=np.int32) for i, c in enumerate(counts)])
    radii = np.array([species[t][1] for t in toa])
    if at_origin:
        pos = np.zeros((len(toa), 3))
    else:
        pos = _random_positions(rng, lat, radii)
    rot = np.tile(np.eye(3), (len(toa), 1, 1)) if identity_rot else _random_rotations(rng, len(toa))
    omega = float(abs(np.dot(lat[0], np.cross(lat[1], lat[2]))))
    return System(lat, omega, types, toa, pos, rot)


def _cubic(omega: float) -> np.ndarray:
    return np.eye(3) * omega ** (1.0 / 3.0)


def make_config(index: int, n_g_override: Optional[int] = None) -> Workload:
    """The five stand-in workloads (0: tiny, 1: medium, 2: precision, 3: batch, 4: large)."""
    seed = SEED_BASE + index
    if index == 0:
        lat = np.eye(3) * 8.0
        sysm = make_system(seed, lat, [(4, 2.2)], [1], at_origin=True, identity_rot=True)
        ks = [kpoint_list(lat, (0.1, 0.2, 0.3), n_g_override or 200)]
    elif index == 1:
        lat = np.diag([12.0, 13.0, 16.0])
        sysm = make_system(seed, lat, [(8, 2.0), (8, 2.4)], [8, 8])
        ks = [kpoint_list(lat, (0.1, 0.2, 0.3), n_g_override or 3000)]
    elif index == 2:
        lat = _cubic(9600.0)
        sysm = make_system(seed, lat, [(10, 1.9), (10, 2.1), (10, 2.3), (10, 2.5)], [16] * 4)
        ks = [kpoint_list(lat, (0.1, 0.2, 0.3), n_g_override or 12000)]
    elif index == 3:
        lat = _cubic(4800.0)
        sysm = make_system(seed, lat, [(6, 2.0), (8, 2.2), (10, 2.4)], [11, 11, 10])
        rng = np.random.Generator(np.random.PCG64(seed + 1000))
        grid = []
        for i in range(4):
            for j in range(4):
                for k in range(3):
                    grid.append(((2 * (i + 1) - 4 - 1) / 8.0, (2 * (j + 1) - 4 - 1) / 8.0,
                                 (2 * (k + 1) - 3 - 1) / 6.0))
        ngs = rng.integers(2500, 4201, size=len(grid))
        if n_g_override:
            ngs = np.full(len(grid), n_g_override)
        ks = [kpoint_list(lat, kr, int(n)) for kr, n in zip(grid, ngs)]
    elif index == 4:
        lat = _cubic(38400.0)
        sysm = make_system(seed, lat, [(10, 1.9), (10, 2.1), (10, 2.3), (10, 2.5)], [64] * 4)
        ks = [kpoint_list(lat, (0.1, 0.2, 0.3), n_g_override or 20000)]
    else:
        raise ValueError(f"no config {index}")
    return Workload(CONFIG_NAMES[index], sysm, ks)


def shift_energies(sysm: System, sigma: float, types: Optional[Sequence[int]] = None) -> System:
    """The same system with every E_l of the chosen species (default: all)
    raised by sigma, a shift of the energy reference. It turns the species'
    T positive definite once sigma is large enough, the case of Sec. 4.6.2
    (the stand-in radial data draw E_l from [-1, 1], so no species is HPD
    as drawn). Species with a T_override are left as they are."""
    chosen = set(range(len(sysm.types)) if types is None else (int(t) for t in types))
    new = [replace(ty, e_l=ty.e_l + sigma) if (i in chosen and ty.T_override is None) else ty
           for i, ty in enumerate(sysm.types)]
    return replace(sysm, types=new)
