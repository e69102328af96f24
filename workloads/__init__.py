"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module draws positions and orientations and states the scalar parameters
of each workload.  It holds none of the method's arithmetic: each side converts
these raw Cartesian quantities into its own coefficient layout.

Workloads (seeds 1411027800 + id):

1. N = 64 spheres, a = 1, eta = 1/(6 pi), random sequential addition (RSA) in a
   cube at volume fraction 0.05 (side 17.50 a), minimum centre distance 2.5 a,
   orientations uniform on the sphere; V^a = 0.1 p, V^(2s) = 0.05 (pp - I/3),
   trap force F = -0.01 R; truncation l <= 2; dt = 0.1, 100 steps.
2. N = 1024, same generator at volume fraction 0.05 (side 44.1 a), truncation l <= 3.
3. N = 10^4 trap: Gaussian cloud sigma = 20 a (no exclusion), k = 0.01,
   V^a = 0.1 p, s0 = 0.05, d0 = 0, superposition, dt = 0.05.
4. 256 independent suspensions, N log-uniform in [32, 4096], volume fraction
   uniform in [0.01, 0.2]; RSA at 2.5 a when it fills, else a jittered cubic lattice.
5. N = 10^5 at volume fraction 0.1 (side 161.2 a), RSA at 2.05 a; force- and
   torque-free (no trap), V^a = 0.1 p, V^(2s) = 0.05 (pp - I/3).
6. Near-field training sets: independent 2- and 3-sphere systems, every sphere
   within [2.05 a, 4 a) of an earlier one and no two closer than 2.05 a,
   orientations uniform (seeds 1411027800 + 6000 + k).

The paper's own runs (10^4 squirmers in a trap, O(10^5) stresslet
superposition) used PyStokes; no dataset exists, so these seeded clouds stand
in for them with the same sizes and geometry.
"""
import math

import numpy as np

SEED_BASE = 1411027800
ETA_DEFAULT = 1.0 / (6.0 * math.pi)


def unit_vectors(n, rng):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def cube_side(N, phi, a=1.0):
    return (N * 4.0 * math.pi * a ** 3 / 3.0 / phi) ** (1.0 / 3.0)


def rsa_cube(N, side, dmin, rng, max_tries=10 ** 6):
    """Random sequential addition in [-side/2, side/2]^3; None if it jams."""
    ncell = max(1, int(side // dmin))
    h = side / ncell
    grid = {}
    pts = np.empty((N, 3))
    tries = 0
    k = 0
    batch = rng.uniform(-side / 2, side / 2, size=(4096, 3))
    bi = 0
    while k < N:
        if bi == len(batch):
            batch = rng.uniform(-side / 2, side / 2, size=(4096, 3))
            bi = 0
        x = batch[bi]
        bi += 1
        tries += 1
        if tries > max_tries * max(1, N // 1000 + 1):
            return None
        c = tuple(np.minimum(((x + side / 2) // h).astype(int), ncell - 1))
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in grid.get((c[0] + dx, c[1] + dy, c[2] + dz), ()):
                        if np.sum((pts[j] - x) ** 2) < dmin * dmin:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pts[k] = x
            grid.setdefault(c, []).append(k)
            k += 1
    return pts


def jittered_lattice(N, side, dmin, rng):
    """Simple-cubic lattice filling the cube, random subset of N sites, jitter keeping dmin."""
    m = int(math.ceil(N ** (1.0 / 3.0)))
    spacing = side / m
    jitter = max(0.0, (spacing - dmin) / 2.0)
    g = (np.arange(m) + 0.5) * spacing - side / 2
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sel = rng.choice(len(sites), size=N, replace=False)
    return sites[sel] + rng.uniform(-jitter, jitter, size=(N, 3)) * (1.0 / math.sqrt(3.0))


def suspension(N, phi, dmin, seed, a=1.0):
    """Positions (RSA, lattice fallback) and orientations for one suspension."""
    rng = np.random.default_rng(seed)
    side = cube_side(N, phi, a)
    R = rsa_cube(N, side, dmin * a, rng, max_tries=2000)
    generator = "rsa"
    if R is None:
        R = jittered_lattice(N, side, dmin * a, rng)
        generator = "lattice"
    p = unit_vectors(N, rng)
    return dict(R=R, p=p, side=side, generator=generator)


def trap_params(**over):
    d = dict(a=1.0, eta=ETA_DEFAULT, k=0.01, vs=0.1, s0=0.05, d0=0.0)
    d.update(over)
    return d


def config1():
    s = suspension(64, 0.05, 2.5, SEED_BASE + 1)
    s.update(trap_params(), trunc=2, dt=0.1, steps=100, rtol=1e-10, name="N64_l2_fp64")
    return s


def config2():
    s = suspension(1024, 0.05, 2.5, SEED_BASE + 2)
    s.update(trap_params(), trunc=3, rtol=1e-10, name="N1024_l3_mixed")
    return s


def config3(N=10000):
    rng = np.random.default_rng(SEED_BASE + 3)
    R = rng.normal(scale=20.0, size=(N, 3))
    p = unit_vectors(N, rng)
    d = dict(R=R, p=p, name="N10000_trap_superposition")
    d.update(trap_params(), trunc=2, dt=0.05, steps=10000)
    return d


def config4(nsys=256):
    rng = np.random.default_rng(SEED_BASE + 4)
    Ns = np.round(np.exp(rng.uniform(math.log(32), math.log(4096), size=nsys))).astype(int)
    phis = rng.uniform(0.01, 0.2, size=nsys)
    systems = []
    for i in range(nsys):
        s = suspension(int(Ns[i]), float(phis[i]), 2.5, SEED_BASE + 4000 + i)
        s["phi"] = float(phis[i])
        systems.append(s)
    return dict(systems=systems, name="batched_256", **trap_params(), trunc=2)


def config5(N=100000):
    s = suspension(N, 0.1, 2.05, SEED_BASE + 5)
    s.update(trap_params(k=0.0), trunc=2, name="N%d_phi0.1_nearfield" % N)
    return s


def nearfield_systems(n2, n3, k=0, rmin=2.05, rmax=4.0):
    """n2 two-sphere and n3 three-sphere systems (a = 1) for the near-field network.

    Sphere 0 sits at a random point of a 10 a cube; each later sphere is placed at a
    distance uniform in [rmin, rmax) from a uniformly chosen earlier sphere, in a
    uniform direction, and redrawn while closer than rmin to any sphere.  Returns
    R [Ntot, 3], p [Ntot, 3] and the system offsets (2-sphere systems first)."""
    rng = np.random.default_rng(SEED_BASE + 6000 + k)
    Rs, offs = [], [0]
    for sz, cnt in ((2, n2), (3, n3)):
        for _ in range(cnt):
            pts = [rng.uniform(-5.0, 5.0, size=3)]
            while len(pts) < sz:
                base = pts[rng.integers(len(pts))]
                d = unit_vectors(1, rng)[0]
                q = base + rng.uniform(rmin, rmax) * d
                if all(np.linalg.norm(q - x) >= rmin for x in pts):
                    pts.append(q)
            Rs.extend(pts)
            offs.append(offs[-1] + sz)
    R = np.array(Rs)
    p = unit_vectors(len(R), rng)
    return dict(R=R, p=p, offsets=offs, **trap_params(k=0.0))


def small_cloud(N, seed, phi=0.05, dmin=2.5):
    """Small RSA suspension for tests."""
    s = suspension(N, phi, dmin, SEED_BASE + 100 + seed)
    s.update(trap_params())
    return s
