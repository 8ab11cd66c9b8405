"""Seeded synthetic initial conditions for the N-body workloads.

This module only draws particle sets; it holds none of the tree method's arithmetic,
so both the CUDA path and the CPU oracle may take their inputs from it.

Every generator returns ``(pos, vel, mass, eps)``:
  * ``pos``  -- (n, 3) float64 whose values are exactly representable in FP32
                (the tree works on FP32 positions; the integrator keeps FP64),
  * ``vel``  -- (n, 3) float64,
  * ``mass`` -- (n,) float32 (equal masses 1/n),
  * ``eps``  -- the Plummer softening length of the model.

Units are G = M_total = 1.  The paper's models came from an external generator
that is not available here; these are restatements from the textbook density
profiles (Plummer 1911; Navarro, Frenk & White 1996; Hernquist 1990; an
exponential disk), with velocities by Eddington inversion in the spherical
potential.  They are timing-grade initial conditions, not exact equilibria.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["plummer", "nfw", "andromeda_like", "batch_systems", "serving_requests",
           "to_fp32_grid"]


def to_fp32_grid(pos: np.ndarray) -> np.ndarray:
    """Round positions to FP32 and return them as float64 (exactly FP32-valued)."""
    return np.asarray(pos, dtype=np.float64).astype(np.float32).astype(np.float64)


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def _finish(pos, vel, n):
    """Move to the centre-of-mass frame (equal masses), round positions to FP32."""
    pos = pos - pos.mean(axis=0)
    vel = vel - vel.mean(axis=0)
    mass = np.full(n, 1.0 / n, dtype=np.float32)
    return to_fp32_grid(pos), np.ascontiguousarray(vel), mass


# --------------------------------------------------------------------------- Plummer
def plummer(n: int, seed: int = 1, eps: float = 1.0 / 64.0):
    """Plummer sphere, G = M = a = 1 (Aarseth, Henon & Wielen 1974 sampling).

    Radius by the inverse cumulative mass, r = (u^{-2/3} - 1)^{-1/2}; speed by
    von Neumann rejection on g(q) = q^2 (1 - q^2)^{7/2}, v = q sqrt(2) (1 + r^2)^{-1/4}.
    """
    rng = np.random.default_rng(seed)
    if n == 0:
        return np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.float32), eps
    u = rng.uniform(1e-10, 1.0 - 1e-10, n)
    # cap the rare far outliers at 100 a (they carry ~1e-6 of the mass)
    r = np.minimum(1.0 / np.sqrt(u ** (-2.0 / 3.0) - 1.0), 100.0)
    pos = r[:, None] * _isotropic(rng, n)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = rng.uniform(0.0, 1.0, todo.size)
        yy = rng.uniform(0.0, 0.1, todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    v = q * math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    vel = v[:, None] * _isotropic(rng, n)
    pos, vel, mass = _finish(pos, vel, n)
    return pos, vel, mass, eps


# --------------------------------------------------------------- spherical machinery
class _Spherical:
    """Tabulated spherical model: total mass profile, potential and Eddington f(E)."""

    def __init__(self, r: np.ndarray, rho_tot: np.ndarray, m_extra: np.ndarray | None = None):
        self.r = r
        shell = 4.0 * math.pi * r * r * rho_tot
        m = np.concatenate([[0.0], np.cumsum(0.5 * (shell[1:] + shell[:-1]) * np.diff(r))])
        # the innermost point: mass of a uniform core of density rho(r0)
        m += 4.0 / 3.0 * math.pi * r[0] ** 3 * rho_tot[0]
        if m_extra is not None:
            m = m + m_extra
        self.mass = m
        # relative potential Psi = -Phi = int_r^inf G M(r')/r'^2 dr'  (G = 1)
        g = m / (r * r)
        seg = 0.5 * (g[1:] + g[:-1]) * np.diff(r)
        tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
        self.psi = tail + m[-1] / r[-1]

    def sample_radii(self, rng, rho_c: np.ndarray, n: int) -> np.ndarray:
        r = self.r
        shell = 4.0 * math.pi * r * r * rho_c
        cdf = np.concatenate([[0.0], np.cumsum(0.5 * (shell[1:] + shell[:-1]) * np.diff(r))])
        cdf /= cdf[-1]
        return np.interp(rng.uniform(0.0, 1.0, n), cdf, r)

    def eddington(self, rho_c: np.ndarray, n_e: int = 2048):
        """f(E) for component density rho_c in this potential (Eddington 1916)."""
        r, psi = self.r, self.psi
        drho_dr = np.gradient(rho_c, r)
        dpsi_dr = -self.mass / (r * r)
        drho_dpsi = drho_dr / dpsi_dr
        # Psi decreases with r: reverse so that the abscissa increases
        psi_inc = psi[::-1]
        g_inc = drho_dpsi[::-1]
        e_grid = np.geomspace(psi.min() * 1.0001, psi.max(), n_e)
        t = np.linspace(0.0, 1.0, 257)
        # F(E) = int_0^E (drho/dPsi) dPsi / sqrt(E - Psi) = int_0^sqrt(E) 2 g(E - s^2) ds
        sq = np.sqrt(e_grid)
        s = sq[:, None] * t[None, :]
        vals = 2.0 * np.interp(e_grid[:, None] - s * s, psi_inc, g_inc, left=0.0, right=g_inc[-1])
        big_f = np.trapezoid(vals, s, axis=1)
        f = np.gradient(big_f, e_grid) / (math.sqrt(8.0) * math.pi ** 2)
        f = np.maximum(f, 0.0)
        return e_grid, f

    def sample_speeds(self, rng, rpart: np.ndarray, e_grid, f, nbins: int = 256, nq: int = 512):
        psi_p = np.interp(rpart, self.r, self.psi)
        v = np.empty(rpart.size)
        lp = np.log(psi_p)
        edges = np.quantile(lp, np.linspace(0.0, 1.0, nbins + 1))
        which = np.clip(np.searchsorted(edges, lp, side="right") - 1, 0, nbins - 1)
        q = np.linspace(0.0, 1.0, nq)
        for b in range(nbins):
            sel = np.nonzero(which == b)[0]
            if sel.size == 0:
                continue
            psib = math.exp(0.5 * (edges[b] + edges[b + 1]))
            pdf = q * q * np.interp(psib * (1.0 - q * q), e_grid, f, left=0.0, right=f[-1])
            cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]))])
            if cdf[-1] <= 0.0:
                v[sel] = 0.0
                continue
            cdf /= cdf[-1]
            qs = np.interp(rng.uniform(0.0, 1.0, sel.size), cdf, q)
            v[sel] = qs * np.sqrt(2.0 * psi_p[sel])
        return v


def _nfw_rho(r, rs, rt):
    x = r / rs
    rho = 1.0 / (x * (1.0 + x) ** 2)
    taper = np.where(r > rt, np.exp(-(r - rt) / rs), 1.0)
    return rho * taper


# --------------------------------------------------------------------------- NFW
def nfw(n: int, seed: int = 2, rs: float = 1.0, rt_over_rs: float = 10.0, eps: float | None = None):
    """NFW sphere (concentration c = r_t/r_s = 10), exponentially tapered beyond r_t.

    rho ~ 1/[x (1+x)^2] for r <= r_t and rho_NFW(r) exp(-(r - r_t)/r_s) beyond,
    sampled out to r_t + 16 r_s; total mass 1; isotropic velocities from the
    Eddington distribution function; softening r_s/256.
    """
    if eps is None:
        eps = rs / 256.0
    rng = np.random.default_rng(seed)
    if n == 0:
        return np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.float32), eps
    rt = rt_over_rs * rs
    r = np.geomspace(1e-6 * rs, rt + 16.0 * rs, 1 << 16)
    rho = _nfw_rho(r, rs, rt)
    sph0 = _Spherical(r, rho)
    rho = rho / sph0.mass[-1]  # normalise to total mass 1
    sph = _Spherical(r, rho)
    rp = sph.sample_radii(rng, rho, n)
    pos = rp[:, None] * _isotropic(rng, n)
    e_grid, f = sph.eddington(rho)
    v = sph.sample_speeds(rng, rp, e_grid, f)
    vel = v[:, None] * _isotropic(rng, n)
    pos, vel, mass = _finish(pos, vel, n)
    return pos, vel, mass, eps


# ----------------------------------------------------------------- Andromeda-like
def andromeda_like(n: int, seed: int = 3, eps: float = 0.01,
                   f_bulge: float = 0.03, f_disk: float = 0.05,
                   a_bulge: float = 0.6, r_d: float = 5.4, z_d: float = 0.6,
                   rs_halo: float = 7.6, rt_halo: float = 200.0):
    """Three-component galaxy: Hernquist bulge, exponential disk, tapered NFW halo.

    Equal-mass particles, split by the components' mass fractions.  The disk has
    surface density ~ exp(-R/R_d) (R drawn from Gamma(2, R_d)) and a sech^2(z/z_d)
    vertical profile; it rotates at the circular speed of the enclosed spherical
    mass with a 10 % Gaussian dispersion.  Bulge and halo velocities come from
    Eddington inversion of their densities in the total spherical potential.
    """
    ss = np.random.SeedSequence(seed)
    rb_seed, rd_seed, rh_seed = ss.spawn(3)
    rngb, rngd, rngh = (np.random.default_rng(s) for s in (rb_seed, rd_seed, rh_seed))
    if n == 0:
        return np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.float32), eps
    nb = int(round(f_bulge * n))
    nd = int(round(f_disk * n))
    nh = n - nb - nd
    f_halo = 1.0 - f_bulge - f_disk
    r_out = rt_halo + 16.0 * rs_halo
    r = np.geomspace(1e-5, r_out, 1 << 16)

    rho_h = _nfw_rho(r, rs_halo, rt_halo)
    rho_h *= f_halo / _Spherical(r, rho_h).mass[-1]
    rho_b = a_bulge / (2.0 * math.pi * r * (r + a_bulge) ** 3)
    rho_b = np.where(r <= rt_halo, rho_b, 0.0)
    rho_b *= f_bulge / _Spherical(r, rho_b).mass[-1]
    # disk mass inside cylindrical radius R, used as a spherical enclosed mass
    m_disk = f_disk * (1.0 - (1.0 + r / r_d) * np.exp(-r / r_d))
    sph = _Spherical(r, rho_h + rho_b, m_extra=m_disk)

    # bulge
    rb = sph.sample_radii(rngb, rho_b, nb)
    pos_b = rb[:, None] * _isotropic(rngb, nb)
    eg, fb = sph.eddington(rho_b)
    vel_b = sph.sample_speeds(rngb, rb, eg, fb)[:, None] * _isotropic(rngb, nb)

    # halo
    rh = sph.sample_radii(rngh, rho_h, nh)
    pos_h = rh[:, None] * _isotropic(rngh, nh)
    eg, fh = sph.eddington(rho_h)
    vel_h = sph.sample_speeds(rngh, rh, eg, fh)[:, None] * _isotropic(rngh, nh)

    # disk
    big_r = -r_d * np.log(rngd.uniform(1e-12, 1.0, nd) * rngd.uniform(1e-12, 1.0, nd))
    big_r = np.minimum(big_r, rt_halo)
    phi = rngd.uniform(0.0, 2.0 * math.pi, nd)
    z = z_d * np.arctanh(np.clip(2.0 * rngd.uniform(0.0, 1.0, nd) - 1.0, -0.999999, 0.999999))
    pos_d = np.stack([big_r * np.cos(phi), big_r * np.sin(phi), z], axis=1)
    vc = np.sqrt(np.interp(big_r, r, sph.mass) / np.maximum(big_r, 1e-6))
    sig = 0.1 * vc
    vel_d = np.stack([-vc * np.sin(phi), vc * np.cos(phi), np.zeros(nd)], axis=1)
    vel_d += sig[:, None] * rngd.standard_normal((nd, 3))

    pos = np.concatenate([pos_b, pos_d, pos_h])
    vel = np.concatenate([vel_b, vel_d, vel_h])
    pos, vel, mass = _finish(pos, vel, n)
    return pos, vel, mass, eps


# ----------------------------------------------------------------- batches/streams
def batch_systems(count: int = 64, seed: int = 4, log2_lo: float = 12.0, log2_hi: float = 18.0):
    """Independent systems with N log-uniform in [2^lo, 2^hi], Plummer or NFW by coin.

    Returns a list of dicts ``{"kind", "n", "seed", "pos", "vel", "mass", "eps"}``.
    """
    rng = np.random.default_rng(seed)
    sizes = np.rint(2.0 ** (log2_lo + (log2_hi - log2_lo) * rng.uniform(0.0, 1.0, count))).astype(int)
    kinds = np.where(rng.uniform(0.0, 1.0, count) < 0.5, "plummer", "nfw")
    seeds = rng.integers(1, 2**31 - 1, count)
    out = []
    for k, (n, kind, s) in enumerate(zip(sizes, kinds, seeds)):
        gen = plummer if kind == "plummer" else nfw
        pos, vel, mass, eps = gen(int(n), seed=int(s))
        out.append({"kind": str(kind), "n": int(n), "seed": int(s), "pos": pos, "vel": vel,
                    "mass": mass, "eps": eps})
    return out


def serving_requests(count: int = 512, seed: int = 5, rate: float = 1.0,
                     log2_lo: float = 12.0, log2_hi: float = 20.0, steps_lo: int = 4, steps_hi: int = 32):
    """A Poisson request stream: arrival times (rate per second), N, model kind, steps.

    Returns a list of dicts without particle data; call ``materialise`` to draw one.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, count)
    t = np.cumsum(gaps) - gaps[0]
    sizes = np.rint(2.0 ** (log2_lo + (log2_hi - log2_lo) * rng.uniform(0.0, 1.0, count))).astype(int)
    kinds = np.where(rng.uniform(0.0, 1.0, count) < 0.5, "plummer", "nfw")
    nsteps = rng.integers(steps_lo, steps_hi + 1, count)
    seeds = rng.integers(1, 2**31 - 1, count)
    return [{"arrival": float(a), "n": int(n), "kind": str(k), "steps": int(s), "seed": int(sd)}
            for a, n, k, s, sd in zip(t, sizes, kinds, nsteps, seeds)]


def materialise(req: dict):
    gen = plummer if req["kind"] == "plummer" else nfw
    return gen(req["n"], seed=req["seed"])
