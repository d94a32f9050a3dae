"""Seeded synthetic docked poses (ligand + binding pocket).

The paper scores docked poses of screening compounds against SARS-CoV-2
targets (Section 4) and evaluates on PDBbind complexes (Section 3.1); neither
dataset is available, so complexes with the same shapes stand in for them:

* ligand: a random bonded tree with planar six-membered ring closures, bond
  lengths U[1.33, 1.55] A, non-bonded heavy atoms at least 1.8 A apart, inside
  a sphere of radius R = max(5, 5 + 0.06 (n_lig - 24)) A;
* pocket: atoms uniform in the shell [R - 1, R + 6] A around the ligand
  centroid, at least 1.2 A from every other atom;
* elements C .62 / N .13 / O .17 / S .03 / P .01 / halogen .04; partial charge
  approximately N(0, 0.3) (Irwin-Hall sum of 12 uniforms);
* the whole complex is translated by U[-40, 40]^3 A and rounded to float32;
* no atom pair lies within 1e-5 A^2 of a squared edge cutoff (1.6, 4.5,
  2.24, 5.22 A) so edge sets do not hinge on the last bit.

Only uniform draws and IEEE +, -, *, /, sqrt are used, so the same seed gives
the same bytes on every platform.  Ligand atoms come first in each pose.

Feature columns (19): element one-hot B, C, N, O, P, S, Se, halogen, metal;
hybridisation; heavy valence; hetero valence; partial charge; ligand flag
(+1 ligand / -1 pocket); hydrophobic; aromatic; acceptor; donor; ring.
"""

from __future__ import annotations

import hashlib

import numpy as np

N_FEAT = 19
GUARD_CUTOFFS = (1.6, 4.5, 2.24, 5.22)
GUARD_EPS = 1e-5

_HEX = ((1.0, 0.0), (0.5, None), (-0.5, None), (-1.0, 0.0), (-0.5, "-"), (0.5, "-"))


def _hex_coeffs():
    s = np.sqrt(3.0) / 2.0
    out = []
    for c, t in _HEX:
        if t is None:
            out.append((c, s))
        elif t == "-":
            out.append((c, -s))
        else:
            out.append((c, 0.0))
    return out


_HEXC = _hex_coeffs()


def _unit(rng):
    while True:
        v = rng.random(3) * 2.0 - 1.0
        r2 = float(v @ v)
        if 1e-4 < r2 <= 1.0:
            return v / np.sqrt(r2)


def _perp_unit(rng, d):
    while True:
        w = _unit(rng)
        w = w - (w @ d) * d
        n2 = float(w @ w)
        if n2 > 1e-3:
            return w / np.sqrt(n2)


def _approx_normal(rng):
    return float(rng.random(12).sum() - 6.0)


def _ligand(rng, n_lig, n_rings):
    """Ligand coordinates and bond list in a local frame centred near 0."""
    R = max(5.0, 5.0 + 0.06 * (n_lig - 24))
    R2 = R * R
    n_rings = max(0, min(n_rings, n_lig // 6))
    for _attempt in range(1000):
        pos = np.zeros((n_lig, 3))
        nb = [[] for _ in range(n_lig)]
        ring = np.zeros(n_lig, dtype=bool)
        n = 0

        def ok(p, skip=()):
            if float(p @ p) > R2:
                return False
            if n == 0:
                return True
            d = pos[:n] - p
            d2 = np.einsum("ij,ij->i", d, d)
            if skip:
                d2[list(skip)] = 1e9
            return bool(d2.min() >= 1.8 * 1.8)

        failed = False
        if n_rings > 0:
            b = 1.33 + 0.22 * rng.random()
            u = _unit(rng)
            v = _perp_unit(rng, u)
            c0 = (rng.random(3) * 2.0 - 1.0) * 0.5
            for k, (c, s) in enumerate(_HEXC):
                pos[k] = c0 + b * (c * u + s * v)
            for k in range(6):
                nb[k].append((k + 1) % 6)
                nb[(k + 1) % 6].append(k)
                ring[k] = True
            n = 6
            rings_left = n_rings - 1
        else:
            pos[0] = (rng.random(3) * 2.0 - 1.0) * 0.5
            n = 1
            rings_left = 0
        tree_total = n_lig - n - 6 * rings_left
        per_ring = tree_total // (rings_left + 1) if rings_left >= 0 else tree_total
        since_ring = 0
        while n < n_lig and not failed:
            want_ring = rings_left > 0 and since_ring >= per_ring and n + 6 <= n_lig
            placed = False
            for _try in range(400):
                p = int(rng.integers(0, n))
                cap = 3 if ring[p] else 4
                if len(nb[p]) >= cap:
                    continue
                b = 1.33 + 0.22 * rng.random()
                d = _unit(rng)
                a0 = pos[p] + b * d
                if not want_ring:
                    if ok(a0, skip=(p,)):
                        pos[n] = a0
                        nb[p].append(n)
                        nb[n].append(p)
                        n += 1
                        since_ring += 1
                        placed = True
                        break
                    continue
                w = _perp_unit(rng, d)
                cen = a0 + b * d
                cand = [cen + b * (-c * d + s * w) for c, s in _HEXC]
                good = ok(cand[0], skip=(p,))
                for q in cand[1:]:
                    good = good and ok(q)
                if good:
                    cc = np.array(cand)
                    dd = cc[:, None, :] - cc[None, :, :]
                    pair = np.einsum("ijk,ijk->ij", dd, dd)
                    np.fill_diagonal(pair, 1e9)
                    good = pair.min() >= 1.2 * 1.2
                if good:
                    base = n
                    for k, q in enumerate(cand):
                        pos[base + k] = q
                        ring[base + k] = True
                    for k in range(6):
                        nb[base + k].append(base + (k + 1) % 6)
                        nb[base + (k + 1) % 6].append(base + k)
                    nb[p].append(base)
                    nb[base].append(p)
                    n += 6
                    rings_left -= 1
                    since_ring = 0
                    placed = True
                    break
            if not placed:
                failed = True
        if not failed and n == n_lig:
            return pos, nb, ring
    raise RuntimeError("ligand generation did not converge")


def _pocket(rng, lig, n_pocket, n_lig):
    R = max(5.0, 5.0 + 0.06 * (n_lig - 24))
    r_in, r_out = R - 1.0, R + 6.0
    cen = lig.mean(axis=0)
    allpos = np.zeros((len(lig) + n_pocket, 3))
    allpos[: len(lig)] = lig
    n = len(lig)
    tries = 0
    while n < len(lig) + n_pocket:
        tries += 1
        if tries > 200000:
            raise RuntimeError("pocket generation did not converge")
        q = (rng.random(3) * 2.0 - 1.0) * r_out
        r2 = float(q @ q)
        if r2 < r_in * r_in or r2 > r_out * r_out:
            continue
        p = cen + q
        d = allpos[:n] - p
        if np.einsum("ij,ij->i", d, d).min() < 1.2 * 1.2:
            continue
        allpos[n] = p
        n += 1
    return allpos[len(lig):]


def _near_cutoff_pairs(x32):
    x = x32.astype(np.float64)
    d = x[:, None, :] - x[None, :, :]
    d2 = np.einsum("ijk,ijk->ij", d, d)
    bad = np.zeros(d2.shape, dtype=bool)
    for c in GUARD_CUTOFFS:
        bad |= np.abs(d2 - c * c) < GUARD_EPS
    iu = np.triu_indices(len(x), 1)
    m = bad[iu]
    return list(zip(iu[0][m].tolist(), iu[1][m].tolist()))


def _features(rng, n_lig, n_pocket, nb, ring):
    n = n_lig + n_pocket
    f = np.zeros((n, N_FEAT), dtype=np.float64)
    elem = np.zeros(n, dtype=np.int64)
    for i in range(n):
        u = rng.random()
        if u < 0.62:
            e = 1      # C
        elif u < 0.75:
            e = 2      # N
        elif u < 0.92:
            e = 3      # O
        elif u < 0.95:
            e = 5      # S
        elif u < 0.96:
            e = 4      # P
        else:
            e = 7      # halogen (F, Cl, Br)
        elem[i] = e
    hetero = np.isin(elem, (2, 3, 4, 5))
    for i in range(n):
        f[i, elem[i]] = 1.0
        lig = i < n_lig
        if lig:
            heavy = len(nb[i])
            het = sum(1 for j in nb[i] if hetero[j])
            aro = 1.0 if ring[i] else 0.0
            rng_flag = aro
            hyb = 2.0 if ring[i] else float(1 + rng.integers(0, 3))
        else:
            heavy = int(1 + rng.integers(0, 3))
            het = int(rng.integers(0, 2))
            aro = 1.0 if (elem[i] == 1 and rng.random() < 0.2) else 0.0
            rng_flag = aro
            hyb = 2.0 if aro else float(1 + rng.integers(0, 3))
        f[i, 9] = hyb
        f[i, 10] = float(heavy)
        f[i, 11] = float(het)
        f[i, 12] = 0.3 * _approx_normal(rng)
        f[i, 13] = 1.0 if lig else -1.0
        f[i, 14] = 1.0 if (elem[i] in (1, 7) and het == 0) else 0.0
        f[i, 15] = aro
        f[i, 16] = 1.0 if (elem[i] == 3 or (elem[i] == 2 and rng.random() < 0.5)) else 0.0
        f[i, 17] = 1.0 if ((elem[i] == 2 and rng.random() < 0.6) or
                           (elem[i] == 3 and rng.random() < 0.3)) else 0.0
        f[i, 18] = rng_flag
    return f.astype(np.float32)


def make_pose(seed: int, n_lig_range, n_pocket_range, rings=None):
    """One pose from its own seed: (xyz float32 [N,3], feat float32 [N,19], n_lig)."""
    rng = np.random.default_rng(seed)
    n_lig = int(rng.integers(n_lig_range[0], n_lig_range[1] + 1))
    n_pocket = int(rng.integers(n_pocket_range[0], n_pocket_range[1] + 1))
    if rings is None:
        rings = max(1, min(4, n_lig // 12))
    lig, nb, ring = _ligand(rng, n_lig, rings)
    pocket = _pocket(rng, lig, n_pocket, n_lig)
    shift = (rng.random(3) * 2.0 - 1.0) * 40.0
    pos = np.concatenate([lig, pocket]) + shift
    for _ in range(1000):
        x32 = pos.astype(np.float32)
        bad = _near_cutoff_pairs(x32)
        if not bad:
            break
        for i, j in bad:
            # nudge the later atom of the pair by 0.01 A
            pos[j] += 0.01 * _unit(rng)
    else:
        raise RuntimeError("could not clear near-cutoff pairs")
    nb_all = nb + [[] for _ in range(n_pocket)]
    ring_all = np.concatenate([ring, np.zeros(n_pocket, dtype=bool)])
    feat = _features(rng, n_lig, n_pocket, nb_all, ring_all)
    return pos.astype(np.float32), feat, n_lig


def pack(poses):
    """Pack [(xyz, feat, n_lig), ...] into the batched SoA layout."""
    counts = [len(p[0]) for p in poses]
    atom_off = np.zeros(len(poses) + 1, dtype=np.int32)
    atom_off[1:] = np.cumsum(counts)
    xyz = np.ascontiguousarray(np.concatenate([p[0] for p in poses]).astype(np.float32))
    feat = np.ascontiguousarray(np.concatenate([p[1] for p in poses]).astype(np.float32))
    n_lig = np.array([p[2] for p in poses], dtype=np.int32)
    return dict(xyz=xyz, feat=feat, atom_off=atom_off, n_lig=n_lig)


def make_batch(workload: dict):
    """A batch from a workload recipe (see ``synth.configs.WORKLOADS``)."""
    poses = [make_pose(s, workload["n_lig"], workload["n_pocket"], workload.get("rings"))
             for s in workload["seeds"]]
    return pack(poses)


def digest(batch) -> str:
    """SHA-256 over the packed arrays, to check two machines made the same inputs."""
    h = hashlib.sha256()
    for k in ("atom_off", "n_lig", "xyz", "feat"):
        h.update(np.ascontiguousarray(batch[k]).tobytes())
    return h.hexdigest()


def pose_slice(batch, p):
    """Atoms of pose p: (xyz, feat, n_lig)."""
    a, b = int(batch["atom_off"][p]), int(batch["atom_off"][p + 1])
    return batch["xyz"][a:b], batch["feat"][a:b], int(batch["n_lig"][p])


def subset(batch, idx):
    """A new packed batch holding the poses idx (in that order)."""
    return pack([pose_slice(batch, int(p)) for p in idx])


def _rotation(rng):
    """Uniform random rotation from a unit quaternion drawn by rejection in the 4-ball."""
    while True:
        q = rng.random(4) * 2.0 - 1.0
        n2 = float(q @ q)
        if 1e-4 < n2 <= 1.0:
            break
    w, x, y, z = q / np.sqrt(n2)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def make_pose_group(seed: int, n_rot: int = 10):
    """Docked-pose stand-ins for one ligand: n_rot poses of the same ligand in the same pocket.

    Ligand heavy-atom count log-normal with median 32 (clipped to 8..90); pocket
    U[150, 1000] atoms.  Pose r rotates the ligand rigidly about its centroid by
    a uniform random rotation and jitters each ligand atom by approximately
    N(0, 0.5^2) A per axis.  Returns [(xyz, feat, n_lig)] * n_rot.
    """
    rng = np.random.default_rng(seed)
    z = _approx_normal(rng)
    n_lig = int(np.clip(np.rint(32.0 * np.exp(0.45 * z)), 8, 90))
    n_pocket = int(rng.integers(150, 1001))
    rings = max(1, min(4, n_lig // 12))
    lig, nb, ring = _ligand(rng, n_lig, rings)
    pocket = _pocket(rng, lig, n_pocket, n_lig)
    shift = (rng.random(3) * 2.0 - 1.0) * 40.0
    nb_all = nb + [[] for _ in range(n_pocket)]
    ring_all = np.concatenate([ring, np.zeros(n_pocket, dtype=bool)])
    feat = _features(rng, n_lig, n_pocket, nb_all, ring_all)
    cen = lig.mean(axis=0)
    out = []
    for _ in range(n_rot):
        R = _rotation(rng)
        jit = np.array([[_approx_normal(rng) for _ in range(3)] for _ in range(n_lig)]) * 0.5
        posed = (lig - cen) @ R.T + cen + jit
        pos = np.concatenate([posed, pocket]) + shift
        for _it in range(1000):
            bad = _near_cutoff_pairs(pos.astype(np.float32))
            if not bad:
                break
            for i, j in bad:
                pos[j] += 0.01 * _unit(rng)
        out.append((pos.astype(np.float32), feat, n_lig))
    return out


def make_uneven_pool(n_groups: int, n_rot: int = 10, seed0: int = 500000, jobs: int = 1):
    """Poses of n_groups ligands x n_rot rotations, in generation order.

    With jobs > 1 the groups are generated in that many worker processes (each group comes from its own seed,
    so the poses and their order are the same); the workers are spawned, so this may run after a CUDA
    context exists in the calling process."""
    if jobs <= 1 or n_groups < 2 * jobs:
        poses = []
        for g in range(n_groups):
            poses.extend(make_pose_group(seed0 + g, n_rot))
        return poses
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    step = (n_groups + 4 * jobs - 1) // (4 * jobs)
    chunks = [(seed0 + g0, min(step, n_groups - g0), n_rot) for g0 in range(0, n_groups, step)]
    poses = []
    with ProcessPoolExecutor(max_workers=jobs, mp_context=mp.get_context("spawn")) as ex:
        for part in ex.map(_pool_chunk, chunks):
            poses.extend(part)
    return poses


def _pool_chunk(args):
    first, count, n_rot = args
    out = []
    for g in range(count):
        out.extend(make_pose_group(first + g, n_rot))
    return out
