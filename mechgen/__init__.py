"""Seeded synthetic inputs: chemical mechanisms and initial fields.

This module is the only code that the CPU oracle (``oracle/``) and the CUDA
library (``paper_2211_03293_gb300``) both consume, and it holds none of the
method's arithmetic: it draws numbers, it never evaluates thermodynamics,
rates, Jacobians or time steps.  The paper's own inputs (the GRI-Mech 3.0
mechanism and a PREMIX flame profile, Sec. 5.1) are not available, so seeded
mechanisms and fields with the same structure stand in for them.

Mechanism recipe (one call of :func:`make_mechanism`):

* species are distinct small element compositions over the element set
  (every single atom first, then random compositions with 1..max_atoms atoms);
  molecular weights follow from standard atomic weights;
* NASA-7 polynomials: cp/R = a1 + c1 t + c2 t^2 + c3 t^3 + c4 t^4, t = T/3000 K,
  a1 ~ U[2.5, 4.5], c1 ~ U[0, 3], c2 ~ U[0, 1.5], c3 ~ U[0, 0.3],
  c4 ~ U[-0.1, 0.1] (positive on 0..6000 K), enthalpy constant
  a6 ~ U[-2000, 2000] K, entropy constant a7 drawn around the value that puts
  the species' standard Gibbs energy near the pressure term at 1000 K;
* reactions conserve elements: a reactant multiset of 1..3 species is drawn,
  every product multiset of 1..3 species with the same element totals (other
  than the reactants themselves) is listed and one is picked uniformly;
  each reaction is written in the direction whose a6 sum does not increase
  (heat-releasing forward direction) and all reactions are reversible;
* Arrhenius: A log-uniform in [1e6, 1e14] in cm-mol-s units, taken as the
  pre-exponential at T_REF = 1000 K (k = A (T/T_REF)^b exp(-Ea/RT), so that b
  does not move k(T_REF) outside the drawn range), converted to SI (m^3, mol, s)
  by (1e-6)^(order-1); b ~ U[-1.5, 1.5]; Ea ~ U[0, 40] kcal/mol, stored as the
  activation temperature Ea/R_u;
* n_thirdbody reactions multiply their rate by [M]; n_troe reactions are
  Lindemann falloff with the 4-parameter Troe broadening (a ~ U[0.1, 0.9],
  T*** ~ U[50, 500], T* ~ U[500, 5000], T** ~ U[2000, 10000] K); the
  low-pressure A0 is A * 1e3 (cm-mol-s) with its own b0 and Ea0 draws;
  every third-body and falloff reaction has its own efficiency row: 1 except
  about three species drawn from U[0.4, 12].

The binary blob written by :meth:`Mechanism.to_blob` is the interface both
sides parse with their own readers.  Layout (little endian, 8-byte aligned
sections): magic ``MRIMECH1``; int32 header [Ns, R, E, n_eff, n_troe, 0, 0, 0];
float64 W[Ns] (kg/mol); float64 nasa[Ns][7]; int32 elem[Ns][E];
int32 rtype[R] (0 plain, 1 third-body, 2 Troe falloff); int32 reac[R][3];
int32 prod[R][3] (species index with repetition for stoichiometry, -1 pad);
int32 eff_row[R]; int32 troe_row[R]; float64 A[R], b[R], Ta[R];
float64 eff[n_eff][Ns]; float64 troe[n_troe][7] = (A0, b0, Ta0, a, T***, T*, T**).
Each int32 section is padded with zeros to a multiple of 8 bytes.
"""
from __future__ import annotations

import dataclasses
import itertools
import struct

import numpy as np

R_U = 8.314462618          # J/(mol K)
KCAL = 4184.0               # J/kcal
P_ATM = 101325.0            # Pa
T_REF = 1000.0              # K, reference temperature of the Arrhenius draw

ATOMIC_WEIGHT = {"H": 1.008e-3, "C": 12.011e-3, "N": 14.007e-3, "O": 15.999e-3}  # kg/mol

MAGIC = b"MRIMECH1"


@dataclasses.dataclass
class Mechanism:
    elements: list
    elem: np.ndarray        # [Ns, E] int32 atom counts
    W: np.ndarray           # [Ns] kg/mol
    nasa: np.ndarray        # [Ns, 7]
    rtype: np.ndarray       # [R] int32
    reac: np.ndarray        # [R, 3] int32 (-1 pad)
    prod: np.ndarray        # [R, 3] int32 (-1 pad)
    eff_row: np.ndarray     # [R] int32 (-1 none)
    troe_row: np.ndarray    # [R] int32 (-1 none)
    A: np.ndarray           # [R] SI
    b: np.ndarray           # [R]
    Ta: np.ndarray          # [R] K
    eff: np.ndarray         # [n_eff, Ns]
    troe: np.ndarray        # [n_troe, 7]
    seed: int = 0

    @property
    def n_species(self) -> int:
        return int(self.W.shape[0])

    @property
    def n_reactions(self) -> int:
        return int(self.A.shape[0])

    @property
    def n(self) -> int:
        """Unknowns per cell: species mass fractions plus temperature."""
        return self.n_species + 1

    def to_blob(self) -> bytes:
        def i32(a):
            raw = np.ascontiguousarray(a, dtype="<i4").tobytes()
            return raw + b"\0" * ((-len(raw)) % 8)

        def f64(a):
            return np.ascontiguousarray(a, dtype="<f8").tobytes()

        Ns, R = self.n_species, self.n_reactions
        hdr = struct.pack("<8i", Ns, R, len(self.elements), self.eff.shape[0],
                          self.troe.shape[0], 0, 0, 0)
        parts = [MAGIC, hdr, f64(self.W), f64(self.nasa), i32(self.elem),
                 i32(self.rtype), i32(self.reac), i32(self.prod),
                 i32(self.eff_row), i32(self.troe_row),
                 f64(self.A), f64(self.b), f64(self.Ta),
                 f64(self.eff.reshape(-1)), f64(self.troe.reshape(-1))]
        return b"".join(parts)


def _species(rng, elements, n_species, max_atoms, max_count):
    E = len(elements)
    comps = [tuple(int(i == e) for i in range(E)) for e in range(E)]
    seen = set(comps)
    tries = 0
    while len(comps) < n_species:
        tries += 1
        if tries > 100000:
            raise RuntimeError("cannot draw enough distinct species")
        natoms = int(rng.integers(2, max_atoms + 1))
        c = [0] * E
        for _ in range(natoms):
            e = int(rng.integers(0, E))
            c[e] += 1
        if any(c[e] > max_count[e] for e in range(E)):
            continue
        t = tuple(c)
        if t in seen:
            continue
        seen.add(t)
        comps.append(t)
    elem = np.array(comps[:n_species], dtype=np.int32)
    W = elem @ np.array([ATOMIC_WEIGHT[e] for e in elements])
    return elem, W


def _nasa(rng, Ns):
    nasa = np.zeros((Ns, 7))
    tau = 3000.0
    a1 = rng.uniform(2.5, 4.5, Ns)
    c1 = rng.uniform(0.0, 3.0, Ns)
    c2 = rng.uniform(0.0, 1.5, Ns)
    c3 = rng.uniform(0.0, 0.3, Ns)
    c4 = rng.uniform(-0.1, 0.1, Ns)
    nasa[:, 0] = a1
    nasa[:, 1] = c1 / tau
    nasa[:, 2] = c2 / tau ** 2
    nasa[:, 3] = c3 / tau ** 3
    nasa[:, 4] = c4 / tau ** 4
    nasa[:, 5] = rng.uniform(-2000.0, 2000.0, Ns)
    # centre of the a7 draw: the value that makes the lnT and constant parts of
    # the species' g/RT equal ln(p_atm / (R_u T)) at T = 1000 K
    lnT0 = np.log(1000.0)
    centre = a1 * (1.0 - lnT0) + lnT0 - np.log(P_ATM / R_U)
    nasa[:, 6] = centre + rng.uniform(-2.0, 2.0, Ns)
    return nasa


def _multisets(Ns, kmax):
    out = []
    for k in range(1, kmax + 1):
        out.extend(itertools.combinations_with_replacement(range(Ns), k))
    return out


def make_mechanism(seed: int, n_species: int, n_reactions: int, elements=("H", "O", "N"),
                   n_thirdbody: int = 0, n_troe: int = 0, max_atoms: int = 4,
                   max_count=None) -> Mechanism:
    """Draw one synthetic, element-conserving, reversible mechanism."""
    rng = np.random.default_rng(seed)
    elements = list(elements)
    E = len(elements)
    if max_count is None:
        max_count = [3] * E
    elem, W = _species(rng, elements, n_species, max_atoms, max_count)
    nasa = _nasa(rng, n_species)

    sets = _multisets(n_species, 3)
    totals = {}
    for s in sets:
        key = tuple(elem[list(s)].sum(axis=0))
        totals.setdefault(key, []).append(s)

    reactions = []
    seen = set()
    tries = 0
    while len(reactions) < n_reactions:
        tries += 1
        if tries > 200000:
            raise RuntimeError("cannot draw enough element-conserving reactions")
        k = int(rng.choice([1, 2, 3], p=[0.25, 0.5, 0.25]))
        r = tuple(sorted(int(i) for i in rng.integers(0, n_species, k)))
        key = tuple(elem[list(r)].sum(axis=0))
        cands = [s for s in totals.get(key, []) if s != r]
        if not cands:
            continue
        pr = cands[int(rng.integers(0, len(cands)))]
        # write the reaction in its heat-releasing direction (a6 sum non-increasing)
        if nasa[list(pr), 5].sum() > nasa[list(r), 5].sum():
            r, pr = pr, r
        if (r, pr) in seen or (pr, r) in seen:
            continue
        seen.add((r, pr))
        reactions.append((r, pr))

    R = n_reactions
    reac = -np.ones((R, 3), np.int32)
    prod = -np.ones((R, 3), np.int32)
    for i, (r, pr) in enumerate(reactions):
        reac[i, :len(r)] = r
        prod[i, :len(pr)] = pr
    nreac = (reac >= 0).sum(axis=1)
    nprod = (prod >= 0).sum(axis=1)

    rtype = np.zeros(R, np.int32)
    small = [i for i in range(R) if nreac[i] <= 2 and nprod[i] <= 2]
    rest = [i for i in range(R) if i not in small]
    order = list(rng.permutation(small)) + list(rng.permutation(rest))
    tb = order[:n_thirdbody]
    fo = order[n_thirdbody:n_thirdbody + n_troe]
    for i in tb:
        rtype[i] = 1
    for i in fo:
        rtype[i] = 2

    # A is the rate coefficient's pre-exponential at T_REF: k = A (T/T_REF)^b exp(-Ea/RT);
    # it is stored in the plain form A' T^b with A' = A / T_REF^b
    A_cgs = 10.0 ** rng.uniform(6.0, 14.0, R)
    b = rng.uniform(-1.5, 1.5, R)
    Ta = rng.uniform(0.0, 40.0, R) * KCAL / R_U
    order_k = nreac + (rtype == 1)
    A = A_cgs * (1e-6) ** (order_k - 1) / T_REF ** b

    eff_row = -np.ones(R, np.int32)
    troe_row = -np.ones(R, np.int32)
    effl, troel = [], []
    for i in sorted(tb + fo):
        row = np.ones(n_species)
        picks = rng.choice(n_species, size=min(3, n_species), replace=False)
        row[picks] = rng.uniform(0.4, 12.0, len(picks))
        eff_row[i] = len(effl)
        effl.append(row)
        if rtype[i] == 2:
            b0 = rng.uniform(-1.5, 1.5)
            A0 = A_cgs[i] * 1e3 * (1e-6) ** (nreac[i]) / T_REF ** b0      # order nreac + 1
            Ta0 = rng.uniform(0.0, 40.0) * KCAL / R_U
            a = rng.uniform(0.1, 0.9)
            T3 = rng.uniform(50.0, 500.0)
            T1 = rng.uniform(500.0, 5000.0)
            T2 = rng.uniform(2000.0, 10000.0)
            troe_row[i] = len(troel)
            troel.append([A0, b0, Ta0, a, T3, T1, T2])
    eff = np.array(effl).reshape(-1, n_species)
    troe = np.array(troel).reshape(-1, 7)
    return Mechanism(elements, elem, W, nasa, rtype, reac, prod, eff_row, troe_row,
                     A, b, Ta, eff, troe, seed)


# ----------------------------------------------------------------------------- fields

def _dirichlet(rng, ncell, Ns):
    return rng.dirichlet(np.ones(Ns), size=ncell)


def field_1d_tanh(seed: int, nx: int, Ns: int, dx: float, T_lo=300.0, T_hi=1800.0, width_cells=4.0):
    """Periodic 1-D line: double-tanh hot band between x = L/4 and 3L/4, Dirichlet(1) Y."""
    rng = np.random.default_rng(seed)
    L = nx * dx
    x = (np.arange(nx) + 0.5) * dx
    w = width_cells * dx
    T = T_lo + (T_hi - T_lo) * 0.5 * (np.tanh((x - L / 4) / w) - np.tanh((x - 3 * L / 4) / w))
    Y = _dirichlet(rng, nx, Ns)
    y = np.concatenate([Y, T[:, None]], axis=1)
    return np.ascontiguousarray(y), np.full(nx, P_ATM)


def field_3d_hotspots(seed: int, nx: int, ny: int, nz: int, Ns: int, dx: float, nspots=8,
                      T_lo=300.0, T_hi=2500.0, amp=(1000.0, 2200.0)):
    """Periodic box: T = 300 K + sum of Gaussian hot spots (sigma in [2dx, 6dx]),
    clipped to [T_lo, T_hi]; Dirichlet(1) mass fractions per cell.  Cell index is
    (k * ny + j) * nx + i."""
    rng = np.random.default_rng(seed)
    L = np.array([nx, ny, nz]) * dx
    centres = rng.uniform(0, 1, (nspots, 3)) * L
    sig = rng.uniform(2 * dx, 6 * dx, nspots)
    A = rng.uniform(amp[0], amp[1], nspots)
    zz, yy, xx = np.meshgrid((np.arange(nz) + 0.5) * dx, (np.arange(ny) + 0.5) * dx,
                             (np.arange(nx) + 0.5) * dx, indexing="ij")
    T = np.full(xx.shape, T_lo)
    for s in range(nspots):
        d = []
        for coord, c, Ld in ((xx, centres[s, 0], L[0]), (yy, centres[s, 1], L[1]), (zz, centres[s, 2], L[2])):
            dd = np.abs(coord - c)
            d.append(np.minimum(dd, Ld - dd))
        r2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
        T += A[s] * np.exp(-r2 / (2 * sig[s] ** 2))
    T = np.clip(T, T_lo, T_hi).reshape(-1)
    ncell = nx * ny * nz
    Y = _dirichlet(rng, ncell, Ns)
    y = np.concatenate([Y, T[:, None]], axis=1)
    return np.ascontiguousarray(y), np.full(ncell, P_ATM)


def field_3d_front(seed: int, nx: int, ny: int, nz: int, Ns: int, dx: float,
                   T_lo=300.0, T_hi=2300.0, width_cells=8.0):
    """Periodic box with a planar flame front in x (double tanh so the field is
    periodic), Dirichlet(1) mass fractions per cell."""
    rng = np.random.default_rng(seed)
    L = nx * dx
    x = (np.arange(nx) + 0.5) * dx
    w = width_cells * dx
    Tx = T_lo + (T_hi - T_lo) * 0.5 * (np.tanh((x - L / 4) / w) - np.tanh((x - 3 * L / 4) / w))
    T = np.broadcast_to(Tx[None, None, :], (nz, ny, nx)).reshape(-1)
    ncell = nx * ny * nz
    Y = _dirichlet(rng, ncell, Ns)
    y = np.concatenate([Y, T[:, None]], axis=1)
    return np.ascontiguousarray(y), np.full(ncell, P_ATM)


# ----------------------------------------------------------------------------- configs

@dataclasses.dataclass
class Workload:
    name: str
    mech: Mechanism
    y0: np.ndarray          # [ncell, n]
    p: np.ndarray           # [ncell]
    grid: dict              # nx, ny, nz, dx, u (3), D, order
    method: int             # 2 = SDIRK2, 3 = SDIRK3
    H: float
    h: float
    n_slow_steps: int
    newton_rtol: float
    ramp: int               # start-up substep levels for the first fast stage of a run


MECH_SMALL = dict(n_species=9, n_reactions=21, elements=("H", "O", "N"), n_thirdbody=2, n_troe=2,
                  max_atoms=4, max_count=[3, 3, 2])
MECH_MEDIUM = dict(n_species=40, n_reactions=170, elements=("C", "H", "O", "N"), n_thirdbody=12,
                   n_troe=8, max_atoms=6, max_count=[2, 4, 3, 2])
MECH_LARGE = dict(n_species=80, n_reactions=350, elements=("C", "H", "O", "N"), n_thirdbody=24,
                  n_troe=16, max_atoms=8, max_count=[3, 6, 3, 2])


@dataclasses.dataclass
class ReactorBatch:
    """Independent constant-pressure 0-D reactors on several mechanisms, advanced
    together over one interval Hstage with fast substeps of about h (no slow
    forcing: K = 0)."""
    groups: list            # [(Mechanism, y0 [ncell, n], p [ncell])]
    method: int
    Hstage: float
    h: float
    newton_rtol: float
    ramp: int


def reactor_batch(seed: int = 0, n_reactors: int = 4096, T_range=(1000.0, 2200.0)) -> ReactorBatch:
    """4096 0-D reactors split evenly over a 9-species / 21-reaction, a 40 / 170 and
    an 80 / 350 mechanism (the last two with third-body and falloff reactions);
    T uniform in T_range, p in [0.5, 2] atm, Dirichlet(1) mass fractions."""
    rng = np.random.default_rng(6000 + seed)
    specs = [(1000 + seed, MECH_SMALL), (3000 + seed, MECH_MEDIUM), (5000 + seed, MECH_LARGE)]
    sizes = [n_reactors // 3 + (1 if i < n_reactors % 3 else 0) for i in range(3)]
    groups = []
    for (mseed, spec), nc in zip(specs, sizes):
        mech = make_mechanism(mseed, **spec)
        Y = _dirichlet(rng, nc, mech.n_species)
        T = rng.uniform(T_range[0], T_range[1], nc)
        p = P_ATM * rng.uniform(0.5, 2.0, nc)
        groups.append((mech, np.ascontiguousarray(np.concatenate([Y, T[:, None]], axis=1)), p))
    return ReactorBatch(groups, 3, 1e-7, 1e-8, 1e-10, 12)


def workload(name: str, seed: int = 0, cells_per_side: int | None = None) -> Workload:
    """The synthetic workloads.  ``line64``: 64-cell periodic line, 9 species /
    21 reactions, 2nd-order slow stencil, SDIRK2, h = H/100, H = 1e-7 s, 10 slow
    steps.  ``box32``: 32^3 periodic box, 40 species / 170 reactions (12
    third-body, 8 falloff), 4th-order slow stencil, SDIRK3, Newton tolerance
    1e-10, H = 5e-8 s, h = H/10, 20 slow steps (``cells_per_side`` shrinks it for
    tests).  ``box64``: the same at 64^3.  ``front128``: the same mechanism and
    method on a 128^3 box with a planar flame front in x (300 -> 2300 K, width 8
    cells), where the per-cell Newton and Jacobian counts vary widely."""
    if name == "line64":
        mech = make_mechanism(1000 + seed, **MECH_SMALL)
        nx = cells_per_side or 64
        dx = 1e-4
        y0, p = field_1d_tanh(2000 + seed, nx, mech.n_species, dx)
        grid = dict(nx=nx, ny=1, nz=1, dx=dx, u=(1.0, 0.0, 0.0), D=1e-5, order=2)
        return Workload(name, mech, y0, p, grid, 2, 1e-7, 1e-9, 10, 1e-10, 10)
    if name == "front128":
        mech = make_mechanism(3000 + seed, **MECH_MEDIUM)
        m = cells_per_side or 128
        dx = 1e-4
        y0, p = field_3d_front(5000 + seed, m, m, m, mech.n_species, dx)
        grid = dict(nx=m, ny=m, nz=m, dx=dx, u=(1.0, 1.0, 1.0), D=1e-5, order=4)
        return Workload(name, mech, y0, p, grid, 3, 5e-8, 5e-9, 20, 1e-10, 16)
    if name in ("box32", "box64"):
        mech = make_mechanism(3000 + seed, **MECH_MEDIUM)
        m = cells_per_side or (32 if name == "box32" else 64)
        dx = 1e-4
        y0, p = field_3d_hotspots(4000 + seed, m, m, m, mech.n_species, dx)
        grid = dict(nx=m, ny=m, nz=m, dx=dx, u=(1.0, 1.0, 1.0), D=1e-5, order=4)
        return Workload(name, mech, y0, p, grid, 3, 5e-8, 5e-9, 20, 1e-10, 16)
    raise KeyError(name)


def random_forcing(seed: int, ncell: int, n: int, K: int, scale_Y=1e2, scale_T=1e5):
    """Seeded slow-forcing coefficients phi[ncell][K][n] of the size a slow
    transport operator produces (|phi_Y| ~ 1e2 1/s, |phi_T| ~ 1e5 K/s)."""
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((ncell, K, n))
    phi[:, :, :-1] *= scale_Y
    phi[:, :, -1] *= scale_T
    # forcing of the mass fractions sums to zero, as a transport operator's does
    phi[:, :, :-1] -= phi[:, :, :-1].mean(axis=2, keepdims=True)
    return np.ascontiguousarray(phi)
