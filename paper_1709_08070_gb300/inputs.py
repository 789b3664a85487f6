"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module holds no arithmetic of the method itself: it only draws random
numbers (charge positions and values, atom chains, node clouds, vectors) with
numpy's seeded generators.  Everything the method computes from these inputs
is done separately by the CUDA library and by the oracle.
"""
import math

import numpy as np

# Seeds of the five standard workloads (Born sphere, Kirkwood sphere, 2,000-atom
# globule, batch of 64 globules, learned warm start), one per workload.
SEED_BORN = 1709080701
SEED_KIRKWOOD = 1709080702
SEED_PROTEIN = 1709080703
SEED_BATCH = 1709080704
SEED_LEARNED = 1709080705


def kirkwood_charges(n=50, ball_radius=16.0, seed=SEED_KIRKWOOD):
    """n charges of +-1 (random signs) uniform in a ball of the given radius."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = ball_radius * rng.random(n) ** (1.0 / 3.0)
    z = u * r[:, None]
    q = rng.choice([-1.0, 1.0], size=n)
    return z, q


def random_vector(n, seed=0, scale=1.0):
    """Gaussian test vector of length n."""
    return scale * np.random.default_rng(seed).standard_normal(n)


def random_rows(n_total, n_rows, seed=0):
    """Sorted distinct row indices for sampled checks."""
    rng = np.random.default_rng(seed)
    n_rows = min(n_rows, n_total)
    return np.sort(rng.choice(n_total, size=n_rows, replace=False)).astype(np.int64)


def sphere_cloud(n, radius=10.0, jitter=0.0, seed=0, weight_range=(0.01, 0.06)):
    """A node cloud for operator checks on caller-given geometry: n points
    uniformly on a sphere (optionally jittered radially), outward unit normals,
    positive random weights.  Points are ordered by a coarse spatial key so
    that neighbouring indices are close in space."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = radius + jitter * rng.standard_normal(n)
    xs = u * r[:, None]
    w = rng.uniform(weight_range[0], weight_range[1], size=n)
    key = np.lexsort((np.floor(u[:, 0] * 8), np.floor(u[:, 1] * 8), np.floor(u[:, 2] * 8)))
    return xs[key], u[key], w[key]


def bisection_order(xs):
    """Permutation that orders points by recursive coordinate bisection: each
    range of n points is split across the longest side of its bounding box,
    the left part a multiple of B points (B = 1024 for n >= 2048, 256 for
    n >= 512, else 32; about half the range), down to 32 points, so that
    aligned runs of 32, 256 and 1024 indices are compact (input preparation
    for caller-ordered clouds; ties broken by the original index)."""
    xs = np.asarray(xs, dtype=np.float64)
    perm = np.arange(xs.shape[0])
    stack = [(0, xs.shape[0])]
    while stack:
        lo, hi = stack.pop()
        n = hi - lo
        if n <= 32:
            continue
        B = 1024 if n >= 2048 else (256 if n >= 512 else 32)
        k = B * max(1, int(math.floor(n / (2.0 * B) + 0.5)))
        seg = xs[perm[lo:hi]]
        ax = int(np.argmax(seg.max(axis=0) - seg.min(axis=0)))
        order = np.lexsort((perm[lo:hi], seg[:, ax]))
        perm[lo:hi] = perm[lo:hi][order]
        stack.append((lo + k, hi))
        stack.append((lo, lo + k))
    return perm


def compact_sphere_cloud(n, radius=10.0, seed=0, weight_range=(0.01, 0.06)):
    """sphere_cloud(n, radius) reordered by bisection_order, so that aligned
    blocks of consecutive indices are compact patches of the sphere."""
    xs, u, w = sphere_cloud(n, radius=radius, seed=seed, weight_range=weight_range)
    perm = bisection_order(xs)
    return xs[perm], u[perm], w[perm]


def sphere_cluster_cloud(n_per, centres, radius=5.0, seed=0, weight_range=(0.01, 0.06)):
    """Several node spheres (n_per points each, the given centres and radius),
    concatenated and ordered by bisection_order: a caller-ordered cloud whose
    parts are far apart compared with a 1024-node tile."""
    parts = []
    for q, c in enumerate(np.asarray(centres, dtype=np.float64)):
        xs, u, w = sphere_cloud(n_per, radius=radius, seed=seed + q, weight_range=weight_range)
        parts.append((xs + c[None, :], u, w))
    xs = np.concatenate([a for a, _, _ in parts])
    u = np.concatenate([b for _, b, _ in parts])
    w = np.concatenate([c for _, _, c in parts])
    perm = bisection_order(xs)
    return xs[perm], u[perm], w[perm]


def globule_atoms(n_atoms, seed=SEED_PROTEIN, step=3.8, min_dist=3.0, beta=100.0, n_cand=128,
                  radius_range=(1.2, 1.9), charge_range=(-0.8, 0.8)):
    """Seeded self-avoiding random-walk chain compacted into a globule:
    bond length `step` A, non-bonded distances >= `min_dist` A.  Each new bead
    is drawn from `n_cand` random bond directions that keep the chain
    self-avoiding, with probability proportional to exp(-beta * (distance to the
    chain's centre of mass - the smallest such distance)), which packs the
    chain towards its centre (at the default beta almost always the most
    central admissible candidate); a walk with no admissible candidate backs
    up 8 beads.  Radii uniform in `radius_range`; partial charges uniform in
    `charge_range` shifted to a net charge of zero.
    Returns (centres (n,3) about their mean, radii, charges)."""
    rng = np.random.default_rng(seed)
    cell = step + min_dist  # every bead that can clash with a candidate is in a neighbouring cell
    pos = np.zeros((n_atoms, 3))
    grid = {}

    def key(p):
        return (int(np.floor(p[0] / cell)), int(np.floor(p[1] / cell)), int(np.floor(p[2] / cell)))

    def near(p, i):
        k = key(p)
        out = []
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    out.extend(grid.get((k[0] + dx, k[1] + dy, k[2] + dz), ()))
        return [j for j in out if j != i - 1]

    grid.setdefault(key(pos[0]), []).append(0)
    csum = pos[0].copy()
    i = 1
    while i < n_atoms:
        d = rng.standard_normal((n_cand, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        cand = pos[i - 1] + step * d
        nb = near(pos[i - 1], i)
        if nb:
            diff = cand[:, None, :] - pos[nb][None, :, :]
            good = np.nonzero(((diff * diff).sum(axis=2) >= min_dist * min_dist).all(axis=1))[0]
        else:
            good = np.arange(n_cand)
        if good.size == 0:
            for _b in range(min(8, i - 1)):
                i -= 1
                grid[key(pos[i])].remove(i)
                csum -= pos[i]
            continue
        cen = csum / i
        dist = np.linalg.norm(cand[good] - cen, axis=1)
        wgt = np.exp(-beta * (dist - dist.min()))
        j = good[rng.choice(good.size, p=wgt / wgt.sum())]
        pos[i] = cand[j]
        grid.setdefault(key(cand[j]), []).append(i)
        csum += cand[j]
        i += 1
    radii = rng.uniform(radius_range[0], radius_range[1], size=n_atoms)
    q = rng.uniform(charge_range[0], charge_range[1], size=n_atoms)
    q -= q.mean()
    return pos - pos.mean(axis=0), radii, q


def residue_atoms(n_atoms, seed=SEED_PROTEIN, atoms_per_residue=8, ca_step=3.8, ca_min=4.5, volume_per_residue=130.0,
                  contact=2.2, radius_range=(1.6, 1.9), charge_range=(-0.8, 0.8)):
    """Seeded heavy-atom-like cloud at protein packing density: a self-avoiding
    chain of residue centres (bond `ca_step` A, non-bonded >= `ca_min` A) grown
    inside a ball of volume n_residues * `volume_per_residue` A^3 (about the
    volume a residue occupies in a folded protein), then `atoms_per_residue` - 1
    further atoms per residue placed 1.5-4 A from its centre, each at least
    `contact` A from every atom placed before it (heavy atoms of real proteins
    overlap their neighbours' van der Waals spheres in the same way).  Radii
    uniform in `radius_range`; charges as in globule_atoms.  Returns
    (centres (n,3) about their mean, radii, charges)."""
    rng = np.random.default_rng(seed)
    n_res = max(1, int(round(n_atoms / atoms_per_residue)))
    R_ball = (3.0 * n_res * volume_per_residue / (4.0 * np.pi)) ** (1.0 / 3.0)
    ca = np.zeros((n_res, 3))
    i = 1
    tries = 0
    while i < n_res:
        d = rng.standard_normal((64, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        cand = ca[i - 1] + ca_step * d
        ok = np.linalg.norm(cand, axis=1) <= R_ball
        if i > 1:
            dd = np.linalg.norm(cand[:, None, :] - ca[None, :i - 1, :], axis=2)
            ok &= (dd >= ca_min).all(axis=1)
        good = np.nonzero(ok)[0]
        if good.size == 0:
            tries += 1
            back = min(i - 1, 4 + tries // 8)
            i -= back
            continue
        ca[i] = cand[good[rng.integers(good.size)]]
        i += 1
    atoms = [c for c in ca]
    cell = {}

    def key(p):
        return tuple(np.floor(p / 4.0).astype(int))

    for j, p in enumerate(atoms):
        cell.setdefault(key(p), []).append(j)

    def clear(p):
        k = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in cell.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                        if np.sum((atoms[j] - p) ** 2) < contact * contact:
                            return False
        return True

    for r in range(n_res):
        placed = 0
        for _ in range(400):
            if placed == atoms_per_residue - 1 or len(atoms) >= n_atoms:
                break
            d = rng.standard_normal(3)
            p = ca[r] + rng.uniform(1.5, 4.0) * d / np.linalg.norm(d)
            if clear(p):
                cell.setdefault(key(p), []).append(len(atoms))
                atoms.append(p)
                placed += 1
    pos = np.array(atoms)
    radii = rng.uniform(radius_range[0], radius_range[1], size=len(pos))
    q = rng.uniform(charge_range[0], charge_range[1], size=len(pos))
    q -= q.mean()
    return pos - pos.mean(axis=0), radii, q


def batch_sizes(n_mol=64, lo=50, hi=3000, seed=SEED_BATCH):
    """Atom counts log-uniform in [lo, hi] and screening constants kappa ~ U[0, 0.2]."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_mol)).round().astype(int)
    kappa = rng.uniform(0.0, 0.2, size=n_mol)
    return n, kappa
