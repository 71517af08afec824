"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no solver arithmetic: it only draws meshes, parameters and
right-hand sides.  It is the one module that both the CUDA path (tests,
bench) and the CPU oracle's tests consume.

Meshes (element lengths h, Sec. 2.2 eq. (Partition)):
  uniform                      h_i = (b-a)/N
  geometric, one-sided         h_{i+1}/h_i = q constant (Sec. 4.3)
  geometric, two-sided         mirrored one-sided halves refined toward both
                               endpoints (ratio q toward each end)
  graded                       x_i = a + (b-a)(i/N)^r (Sec. 5, Example 1)
  graded, two-sided            Example 2's mesh family

Right-hand sides:
  manufactured_rhs  f for a given u written as powers of (x-a): the
                    fractional integral of a power function is a power
                    function, Gamma(mu+1)/Gamma(mu+1+beta) (x-a)^(mu+beta),
                    so -D(I^{2-alpha} u') is a finite sum of powers.
  legendre_rhs      seeded Legendre coefficients decaying like (k+1)^-2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# RHS kinds shared with the C ABI (include/hfsem.h)
RHS_LOAD_VECTOR = 0
RHS_FRAC_POWERS = 1
RHS_LEGENDRE_AB = 2


def mesh_uniform(N: int, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    return np.full(N, (b - a) / N)


def mesh_geometric_one_sided(N: int, q: float, a: float = 0.0,
                             b: float = 1.0) -> np.ndarray:
    """h_{i+1} = q h_i; q < 1 refines toward b, q > 1 toward a."""
    w = q ** np.arange(N, dtype=np.float64)
    return (b - a) * w / w.sum()


def mesh_geometric_two_sided(N: int, q: float, a: float = 0.0,
                             b: float = 1.0) -> np.ndarray:
    """N even; N/2 elements per side, each half graded by ratio q toward its
    endpoint (smallest elements at a and at b)."""
    if N % 2:
        raise ValueError("two-sided geometric mesh needs even N")
    half = q ** np.arange(N // 2 - 1, -1, -1, dtype=np.float64)  # small at a
    h = np.concatenate([half, half[::-1]])
    return (b - a) * h / h.sum()


def mesh_graded(N: int, r: float, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    """x_i = a + (b-a)(i/N)^r, lengths from the difference of powers."""
    i = np.arange(N + 1, dtype=np.float64)
    x = (i / N) ** r
    return (b - a) * np.diff(x)


def mesh_graded_two_sided(N: int, rl: float = 7.0, rr: float = 5.0,
                          a: float = 0.0, b: float = 10.0) -> np.ndarray:
    """Example 2's family: x_i = a + m (2i/N)^rl on the left half and
    x_i = b - m (2(N-i)/N)^rr on the right half, m = (b-a)/2.  (The printed
    right-half formula uses (N-2i)/N, which leaves (a,b) for i > N/2; the
    mirrored grading toward b is read here.)"""
    if N % 2:
        raise ValueError("N even")
    m = 0.5 * (b - a)
    i = np.arange(N // 2 + 1, dtype=np.float64)
    hl = np.diff(m * (2.0 * i / N) ** rl)
    hr = hl_r = np.diff(m * (2.0 * i / N) ** rr)[::-1]
    del hl_r
    return np.concatenate([hl, hr])


def manufactured_rhs(u_coeffs, alpha: float, theta: float, rho: float,
                     a: float, b: float, powers=None):
    """f for the manufactured solution u(x) = sum_k u_k (x-a)^{p_k}.

    powers defaults to 0, 1, 2, ... (a polynomial); non-integer powers are
    allowed only for theta == 1 (the right-sided integral of a non-integer
    power of (x-a) is not a finite sum).  Returns (terms, c1, c2) with terms
    a list of (coef, exponent, side) as used by the FRAC_POWERS RHS kind.

    Weak-form consistent with the boundary lifting: only u' enters the
    fractional terms, so
      f = -theta   sum_k u_k Gamma(p_k+1)/Gamma(p_k+1-alpha) (x-a)^(p_k-alpha)
          -(1-theta) sum_j d_j Gamma(j+1)/Gamma(j+1-alpha)   (b-x)^(j-alpha)
          + rho u,
    where d_j are u's coefficients in powers of (b - x)."""
    u = np.asarray(u_coeffs, dtype=np.float64)
    if powers is None:
        powers = np.arange(len(u), dtype=np.float64)
    powers = np.asarray(powers, dtype=np.float64)
    integer = np.all(powers == np.round(powers))
    if not integer and theta != 1.0:
        raise ValueError("non-integer powers need theta == 1")
    L = b - a
    terms = []
    for uk, pk in zip(u, powers):
        if uk == 0.0:
            continue
        if pk > 0.0 and theta != 0.0:
            terms.append((-theta * uk * math.gamma(pk + 1) / math.gamma(pk + 1 - alpha),
                          pk - alpha, "a"))
        if rho != 0.0:
            terms.append((rho * uk, pk, "a"))
    if theta != 1.0:
        deg = int(powers.max())
        d = np.zeros(deg + 1)
        for uk, pk in zip(u, powers):
            k = int(pk)
            for j in range(k + 1):
                d[j] += uk * math.comb(k, j) * L ** (k - j) * (-1.0) ** j
        for j in range(1, deg + 1):
            if d[j] != 0.0:
                terms.append((-(1.0 - theta) * d[j] * math.gamma(j + 1)
                              / math.gamma(j + 1 - alpha), j - alpha, "b"))
    c1 = float(u[powers == 0].sum()) if np.any(powers == 0) else 0.0
    c2 = float(np.sum(u * L ** powers))
    return terms, c1, c2


def legendre_rhs(K: int, rng: np.random.Generator) -> np.ndarray:
    """f = sum_{k=0}^{K} g_k (k+1)^-2 L_k(xi_[a,b]), g_k ~ N(0, 1)."""
    g = rng.standard_normal(K + 1)
    return g / (np.arange(K + 1, dtype=np.float64) + 1.0) ** 2


@dataclass
class Problem:
    """One instance of -D^2(theta aI^{2-alpha}u + (1-theta) xI^{2-alpha}u)
    + rho u = f on (a, b), u(a) = c1, u(b) = c2, discretised with N elements
    of degree P.  rhs_kind / rhs_data follow the FRAC_POWERS / LEGENDRE_AB /
    LOAD_VECTOR kinds; nrhs right-hand sides."""
    h: np.ndarray
    P: int
    alpha: float
    theta: float
    rho: float
    a: float = 0.0
    b: float = 1.0
    c1: float = 0.0
    c2: float = 0.0
    rhs_kind: int = RHS_LEGENDRE_AB
    rhs: list = field(default_factory=list)   # one entry per RHS
    u_exact: object = None                    # polynomial coeffs in (x-a) if known
                                              # (a list, one per RHS, for several)
    name: str = ""
    arrival: float = 0.0                      # request streams: arrival time
    reuse_of: int = -1                        # request streams: earlier request whose
                                              # mesh and parameters this one repeats

    @property
    def N(self) -> int:
        return len(self.h)

    @property
    def Nd(self) -> int:
        return self.N * self.P - 1


def config1() -> Problem:
    """(0,1), N=16 uniform, P=4, alpha=1.5, theta=0.5, rho=0,
    u = x^2 (1-x)^2, c1 = c2 = 0."""
    alpha, theta, rho = 1.5, 0.5, 0.0
    u = [0.0, 0.0, 1.0, -2.0, 1.0]
    terms, c1, c2 = manufactured_rhs(u, alpha, theta, rho, 0.0, 1.0)
    return Problem(h=mesh_uniform(16), P=4, alpha=alpha, theta=theta, rho=rho,
                   c1=c1, c2=c2, rhs_kind=RHS_FRAC_POWERS, rhs=[terms],
                   u_exact=u, name="C1 uniform N=16 P=4")


def config2(K: int = 32, seed: int = 18080002):
    """Nine instances: N=1024 uniform on (0,1), P=8, rho=1,
    alpha in {1.2,1.5,1.8} x theta in {0,0.3,0.5}, seeded Legendre f."""
    rng = np.random.default_rng(seed)
    out = []
    for alpha in (1.2, 1.5, 1.8):
        for theta in (0.0, 0.3, 0.5):
            out.append(Problem(h=mesh_uniform(1024), P=8, alpha=alpha,
                               theta=theta, rho=1.0,
                               rhs_kind=RHS_LEGENDRE_AB,
                               rhs=[legendre_rhs(K, rng)],
                               name=f"C2 uniform N=1024 P=8 a={alpha} t={theta}"))
    return out


def config3(K: int = 32, seed: int = 18080003) -> Problem:
    """Two-sided geometric q=0.5, N=256, P=16, alpha=1.3, theta=0.7, rho=1."""
    rng = np.random.default_rng(seed)
    return Problem(h=mesh_geometric_two_sided(256, 0.5), P=16, alpha=1.3,
                   theta=0.7, rho=1.0, rhs_kind=RHS_LEGENDRE_AB,
                   rhs=[legendre_rhs(K, rng)],
                   name="C3 geometric-2s q=0.5 N=256 P=16")


def config4(n_inst: int = 512, nrhs: int = 4, seed: int = 18080004):
    """Seeded batch: N~U{32..512}, P~U{2..12}, alpha~U(1.1,1.9),
    theta~U(0,1), rho~U(0,2); meshes uniform / two-sided geometric
    (q~U(0.3,0.7)) / graded r in {2,3}; u = x(1-x)p(x), deg p <= 4."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        N = int(rng.integers(32, 513))
        P = int(rng.integers(2, 13))
        alpha = float(rng.uniform(1.1, 1.9))
        theta = float(rng.uniform(0.0, 1.0))
        rho = float(rng.uniform(0.0, 2.0))
        fam = int(rng.integers(0, 3))
        if fam == 0:
            h, mname = mesh_uniform(N), "uniform"
        elif fam == 1:
            N += N % 2
            q = float(rng.uniform(0.3, 0.7))
            h, mname = mesh_geometric_two_sided(N, q), f"geo2s q={q:.3f}"
        else:
            r = float(rng.integers(2, 4))
            h, mname = mesh_graded(N, r), f"graded r={r:g}"
        rhs = []
        for _ in range(nrhs):
            pc = rng.standard_normal(int(rng.integers(0, 5)) + 1)
            # u = x (1 - x) p(x) as coefficients in powers of x
            u = np.convolve([0.0, 1.0, -1.0], pc)
            terms, _, _ = manufactured_rhs(u, alpha, theta, rho, 0.0, 1.0)
            rhs.append(terms)
        out.append(Problem(h=h, P=P, alpha=alpha, theta=theta, rho=rho,
                           rhs_kind=RHS_FRAC_POWERS, rhs=rhs,
                           name=f"C4[{i}] {mname} N={N} P={P}"))
    return out


def geometric_q_floor(N: int, tiny: float = 1e-280) -> float:
    """Smallest ratio q for which a two-sided geometric mesh of N elements
    keeps its smallest element above tiny relative to the largest (FP64
    underflows near 1e-308)."""
    return tiny ** (1.0 / max(1, N // 2 - 1))


def config5_requests(n: int = 10000, seed: int = 18080005, rate: float = 1.0):
    """Seeded request stream (a generator, meshes drawn as each request is
    produced): Poisson arrivals of the given rate; N_d log-uniform on
    [100, 65535], P~U{2..16}, N = ceil((N_d+1)/P) <= 4096; alpha, theta, rho
    and the mesh family as config 4 (two-sided geometric q raised to
    geometric_q_floor(N) where the drawn q would underflow FP64); nrhs~U{1..16}
    right-hand sides from u = x(1-x)p(x), deg p <= 4 (u_exact holds them);
    30 % of the requests repeat the mesh and parameters (the factor key) of a
    uniformly chosen earlier request, with new right-hand sides."""
    rng = np.random.default_rng(seed)
    t = 0.0
    keys = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        reuse = bool(keys) and rng.uniform() < 0.3
        if reuse:
            j = int(rng.integers(0, len(keys)))
            N, P, alpha, theta, rho, fam, q, r, _ = keys[j]
            src = keys[j][8]
        else:
            Nd = int(round(math.exp(rng.uniform(math.log(100.0), math.log(65535.0)))))
            P = int(rng.integers(2, 17))
            N = min(4096, max(1, -(-(Nd + 1) // P)))
            alpha = float(rng.uniform(1.1, 1.9))
            theta = float(rng.uniform(0.0, 1.0))
            rho = float(rng.uniform(0.0, 2.0))
            fam = int(rng.integers(0, 3))
            q = float(rng.uniform(0.3, 0.7))
            r = float(rng.integers(2, 4))
            if fam == 1:
                N += N % 2
                if N > 4096:
                    N -= 2
                q = max(q, geometric_q_floor(N))
            src = i
            keys.append((N, P, alpha, theta, rho, fam, q, r, i))
        if fam == 0:
            h, mname = mesh_uniform(N), "uniform"
        elif fam == 1:
            h, mname = mesh_geometric_two_sided(N, q), f"geo2s q={q:.3f}"
        else:
            h, mname = mesh_graded(N, r), f"graded r={r:g}"
        nrhs = int(rng.integers(1, 17))
        rhs, us = [], []
        for _ in range(nrhs):
            pc = rng.standard_normal(int(rng.integers(0, 5)) + 1)
            u = np.convolve([0.0, 1.0, -1.0], pc)
            terms, _, _ = manufactured_rhs(u, alpha, theta, rho, 0.0, 1.0)
            rhs.append(terms)
            us.append(u)
        yield Problem(h=h, P=P, alpha=alpha, theta=theta, rho=rho,
                      rhs_kind=RHS_FRAC_POWERS, rhs=rhs, u_exact=us,
                      name=f"C5[{i}] {mname} N={N} P={P} nrhs={nrhs}",
                      arrival=t, reuse_of=(src if reuse else -1))


def config5_max_request(family: str = "graded", nrhs: int = 16, seed: int = 18080055):
    """The largest request of the stream: N = 4096, P = 16 (N_d = 65535),
    uniform (Toeplitz operator) or graded r = 2 (dense operator), nrhs
    manufactured right-hand sides from u = x(1-x)p(x), deg p <= 4."""
    rng = np.random.default_rng(seed)
    N, P = 4096, 16
    alpha = float(rng.uniform(1.1, 1.9))
    theta = float(rng.uniform(0.0, 1.0))
    rho = float(rng.uniform(0.0, 2.0))
    h = mesh_uniform(N) if family == "uniform" else mesh_graded(N, 2.0)
    rhs, us = [], []
    for _ in range(nrhs):
        pc = rng.standard_normal(5)
        u = np.convolve([0.0, 1.0, -1.0], pc)
        terms, _, _ = manufactured_rhs(u, alpha, theta, rho, 0.0, 1.0)
        rhs.append(terms)
        us.append(u)
    return Problem(h=h, P=P, alpha=alpha, theta=theta, rho=rho, rhs_kind=RHS_FRAC_POWERS,
                   rhs=rhs, u_exact=us, name=f"C5 max {family} N={N} P={P} nrhs={nrhs}")
