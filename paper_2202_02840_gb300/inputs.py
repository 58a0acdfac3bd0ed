"""Seeded synthetic inputs for the CRKSPH pair passes.

This module is shared by the CUDA path (bench, tests) and the FP64 oracle
tests, so it holds none of the method's arithmetic: no SPH kernel, no moment,
no force.  Everything is generated in FP64 on the host from numpy's
counter-based Philox generator and stored as FP32, which is what both sides
read.  All workloads live in the periodic unit cube in natural units
(a = 1, adot = 0), with equal masses m = 1/N so the mean density is 1.

Workloads (paper context: Sec. 3.1 hydro tests, Sec. 2.5 initial conditions):
  uniform(16)        jittered lattice (+-0.1 spacing), u = 1, v ~ N(0, 0.01^2)
  sedov(64)          jittered lattice (+-0.05 spacing), u = 1e-6, E = 1 deposited
                     with a smooth compact taper inside 2 spacings of the centre
  zeldovich(128)     lattice displaced by the Zel'dovich approximation of a
                     Gaussian field with P(k) ~ k^-2 (cut at the lattice Nyquist),
                     amplitude bisected so the 99.9th/0.1th percentile ratio of
                     the Lagrangian density 1/|det(I + A dpsi/dq)| is ~1e4;
                     v = A psi; log10 u ~ N(0, 1)
Smoothing lengths: h = n_h * spacing = 4 spacing on lattices; for the
displaced workload h is the distance to the 268th nearest particle (a k-d tree
query, not an SPH sum), which puts the neighbour count near its target.
"""
import numpy as np

N_H = 4.0          # particles per smoothing length used to size h (Sec. 2.6)
N_RES = 268        # target neighbour count quoted with n_h = 4 (Sec. 2.6)


def rng(seed: int) -> np.random.Generator:
    """Counter-based Philox stream for one seed."""
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _to_unit_f32(x: np.ndarray) -> np.ndarray:
    """Wrap FP64 coordinates into [0,1) and store as FP32, keeping them < 1."""
    x = np.mod(x, 1.0)
    f = x.astype(np.float32)
    f[f >= np.float32(1.0)] = np.float32(0.0)
    f[f < 0] = np.float32(0.0)
    return f


def lattice(n_side: int) -> np.ndarray:
    """Cell-centred cubic lattice (i + 1/2) / n_side, x fastest; shape (N, 3)."""
    c = (np.arange(n_side, dtype=np.float64) + 0.5) / n_side
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def jittered_lattice(n_side: int, amp: float, seed: int) -> np.ndarray:
    """Lattice displaced by U(-amp, amp) spacings per axis."""
    q = lattice(n_side)
    d = rng(seed).uniform(-amp, amp, size=q.shape) / n_side
    return np.mod(q + d, 1.0)


def pack(pos: np.ndarray, h, vel: np.ndarray, u, mass) -> dict:
    """FP32 particle records: pos_h (N,4) = x,y,z,h; vel_u (N,4) = vx,vy,vz,u; mass (N,)."""
    n = pos.shape[0]
    pos_h = np.empty((n, 4), np.float32)
    pos_h[:, :3] = _to_unit_f32(pos)
    pos_h[:, 3] = np.broadcast_to(np.asarray(h, np.float64), (n,)).astype(np.float32)
    vel_u = np.empty((n, 4), np.float32)
    vel_u[:, :3] = vel.astype(np.float32)
    vel_u[:, 3] = np.broadcast_to(np.asarray(u, np.float64), (n,)).astype(np.float32)
    m = np.broadcast_to(np.asarray(mass, np.float64), (n,)).astype(np.float32).copy()
    return {"pos_h": pos_h, "vel_u": vel_u, "mass": m}


def uniform(n_side: int = 16, seed_pos: int = 1, seed_vel: int = 2,
            jitter: float = 0.1, sigma_v: float = 0.01, u: float = 1.0) -> dict:
    """Jittered lattice gas at rest up to small Gaussian velocities."""
    n = n_side ** 3
    pos = jittered_lattice(n_side, jitter, seed_pos)
    vel = rng(seed_vel).normal(0.0, sigma_v, size=(n, 3))
    return pack(pos, N_H / n_side, vel, u, 1.0 / n)


def sedov(n_side: int = 64, seed: int = 3, jitter: float = 0.05, u0: float = 1e-6,
          E: float = 1.0, r_dep: float = 2.0) -> dict:
    """Sedov-Taylor blast: cold jittered lattice, energy E deposited around the
    box centre with the taper w = (1 - (r/R)^2)^2 inside R = r_dep spacings."""
    n = n_side ** 3
    pos = jittered_lattice(n_side, jitter, seed)
    m = 1.0 / n
    d = pos - 0.5
    r = np.sqrt((d * d).sum(axis=1))
    R = r_dep / n_side
    w = np.where(r < R, (1.0 - (r / R) ** 2) ** 2, 0.0)
    u = np.full(n, u0) + E * w / (m * w.sum())
    return pack(pos, N_H / n_side, np.zeros((n, 3)), u, m)


def _kvec(n: int):
    k1 = 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n)
    kr = 2.0 * np.pi * np.fft.rfftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(k1, k1, kr, indexing="ij")
    return kx, ky, kz


def zeldovich_fields(n_side: int, seed: int):
    """Displacement psi (3, n,n,n) and the Lagrangian-density invariants of
    T_ab = d psi_a / d q_b for a Gaussian field with P(k) ~ k^-2, k <= pi n."""
    n = n_side
    white = rng(seed).standard_normal((n, n, n))
    wk = np.fft.rfftn(white)
    kx, ky, kz = _kvec(n)
    k2 = kx * kx + ky * ky + kz * kz
    kmag = np.sqrt(k2)
    keep = (k2 > 0) & (kmag <= np.pi * n)
    dk = np.zeros_like(wk)
    dk[keep] = wk[keep] / kmag[keep]                 # sqrt(P) with P ~ k^-2
    inv_k2 = np.zeros_like(k2)
    inv_k2[keep] = 1.0 / k2[keep]
    ks = (kx, ky, kz)
    # psi_k = i k delta_k / k^2  so that delta = -div psi
    psi = np.stack([np.fft.irfftn(1j * ks[a] * dk * inv_k2, s=(n, n, n), axes=(0, 1, 2)) for a in range(3)])
    scale = 1.0 / np.sqrt((psi ** 2).sum(axis=0).mean())   # unit rms displacement
    psi *= scale
    T = np.empty((3, 3, n, n, n))
    for a in range(3):
        for b in range(a, 3):
            T[a, b] = np.fft.irfftn(-ks[a] * ks[b] * dk * inv_k2, s=(n, n, n), axes=(0, 1, 2)) * scale
            T[b, a] = T[a, b]
    I1 = T[0, 0] + T[1, 1] + T[2, 2]
    I2 = (T[0, 0] * T[1, 1] - T[0, 1] * T[1, 0] + T[1, 1] * T[2, 2] - T[1, 2] * T[2, 1]
          + T[0, 0] * T[2, 2] - T[0, 2] * T[2, 0])
    I3 = (T[0, 0] * (T[1, 1] * T[2, 2] - T[1, 2] * T[2, 1])
          - T[0, 1] * (T[1, 0] * T[2, 2] - T[1, 2] * T[2, 0])
          + T[0, 2] * (T[1, 0] * T[2, 1] - T[1, 1] * T[2, 0]))
    return psi, (I1, I2, I3)


def _contrast(A: float, inv) -> float:
    I1, I2, I3 = inv
    det = 1.0 + A * I1 + A * A * I2 + A ** 3 * I3
    rho = 1.0 / np.maximum(np.abs(det), 1e-30)
    lo, hi = np.percentile(rho, [0.1, 99.9])
    return hi / lo


def knn_h(pos: np.ndarray, k: int = N_RES, h_cap: float = 0.3) -> np.ndarray:
    """Distance to the k-th nearest particle (self counted first), periodic."""
    from scipy.spatial import cKDTree
    tree = cKDTree(pos, boxsize=1.0)
    d, _ = tree.query(pos, k=[k], workers=-1)
    return np.minimum(d[:, 0], h_cap)


def zeldovich(n_side: int = 128, seed: int = 4, seed_u: int = 5, contrast: float = 1e4,
              h_cap: float = 0.3) -> dict:
    """Clustered gas: Zel'dovich-displaced lattice with amplitude set by bisection."""
    n = n_side ** 3
    psi, inv = zeldovich_fields(n_side, seed)
    lo, hi = 0.0, 1.0 / n_side
    while _contrast(hi, inv) < contrast:
        hi *= 2.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if _contrast(mid, inv) < contrast:
            lo = mid
        else:
            hi = mid
    A = 0.5 * (lo + hi)
    q = lattice(n_side)
    disp = np.stack([psi[a].ravel() for a in range(3)], axis=1) * A
    pos = np.mod(q + disp, 1.0)
    pos32 = _to_unit_f32(pos).astype(np.float64)
    h = knn_h(pos32, N_RES, h_cap)
    u = 10.0 ** rng(seed_u).normal(0.0, 1.0, size=n)
    out = pack(pos32, h, disp, u, 1.0 / n)
    out["amplitude"] = A
    return out


def sod(n_hi: int = 64) -> dict:
    """Sod shock tube of the paper's Sec. 4 test, scaled into the periodic unit
    cube: the paper's domain x in [0, 2) with interfaces at 0.5 and 1.5 becomes
    x in [0, 1) with interfaces at 1/4 and 3/4 (lengths and times halved, the
    paper's t = 0.15 is t = 0.075 here).  High state rho = P = 1 for x < 1/4 and
    x >= 3/4, low state rho = P = 1/8 between (the same temperature), at rest;
    a step-function start, which the paper reports gives results
    indistinguishable from its smoothed interface.  Equal masses m = 1/n_hi^3:
    the high state is a cubic lattice of spacing 1/n_hi, the low state one of
    spacing 2/n_hi; h = 4 spacings; u = P/((gamma-1) rho) = 3/2 everywhere.
    The isolated half x in [0, 1/2) holds one interface (high on the left)."""
    n = int(n_hi)
    if n % 8 or n < 32:
        raise ValueError("n_hi must be a multiple of 8 and at least 32")
    gamma = 5.0 / 3.0
    hx = (np.concatenate([np.arange(n // 4), np.arange(3 * n // 4, n)]) + 0.5) / n
    ht = (np.arange(n) + 0.5) / n
    lx = 0.25 + (np.arange(n // 4) + 0.5) * 2.0 / n
    lt = (np.arange(n // 2) + 0.5) * 2.0 / n
    hi = np.stack(np.meshgrid(hx, ht, ht, indexing="ij"), -1).reshape(-1, 3)
    lo = np.stack(np.meshgrid(lx, lt, lt, indexing="ij"), -1).reshape(-1, 3)
    x = np.concatenate([hi, lo])
    h = np.concatenate([np.full(len(hi), 4.0 / n), np.full(len(lo), 8.0 / n)])
    vel = np.zeros((len(x), 3))
    u = np.full(len(x), 1.0 / (gamma - 1.0) * 1.0)   # P/rho = 1 on both sides
    st = pack(x, h, vel, u, 1.0 / n ** 3)
    st.update({"t_end": 0.075, "x0": 0.25, "domain": (0.0, 0.5), "left": (1.0, 0.0, 1.0),
               "right": (0.125, 0.0, 0.125), "gamma": gamma})
    return st


def sedov_boxes(nbox: int = 64, side_lo: int = 16, side_hi: int = 96, seed: int = 0) -> dict:
    """Independent Sedov boxes for the batched step: box b is sedov(side_b,
    seed=b) with side_b drawn uniformly from the integers side_lo..side_hi;
    arrays concatenated box-major, box_start[b] = first row of box b."""
    sides = rng(7000 + int(seed)).integers(side_lo, side_hi + 1, nbox)
    parts = [sedov(int(sd), seed=b) for b, sd in enumerate(sides)]
    start = np.cumsum([0] + [p["pos_h"].shape[0] for p in parts])
    out = {k: np.concatenate([p[k] for p in parts]) for k in ("pos_h", "vel_u", "mass")}
    out["box_start"] = [int(x) for x in start]
    out["sides"] = [int(x) for x in sides]
    return out


def mlp_init(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the 8-64-64-1 network, packed as
    [W1 (64x8), b1, W2 (64x64), b2, W3, b3]: fan-in scaled normal hidden
    weights, zero biases and a zero output row (so that the untrained network
    outputs 0 and the proposal starts as its reference).  FP32."""
    r = rng(1000 + int(seed))
    W1 = r.normal(0.0, 1.0 / np.sqrt(8.0), (64, 8))
    W2 = r.normal(0.0, 1.0 / np.sqrt(64.0), (64, 64))
    w = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), np.zeros(64), [0.0]])
    return w.astype(np.float32)


WORKLOADS = {
    "uniform": uniform,
    "sedov": sedov,
    "zeldovich": zeldovich,
}
