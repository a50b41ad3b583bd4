"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the excited-state method: it only draws
molecules (element lists and Cartesian coordinates in Angstrom), per-element
NDDO parameter sets inside physical ranges, and random trial vectors.

The paper (Section "Results and discussion") measures on carbon nanotubes,
dendrimers and perylene-diimide stacks with the AM1 Hamiltonian; neither the
geometries nor the AM1 parameters are available, so seeded chains and a
seeded parameter set stand in for them.

Every geometry is built with IEEE-exact operations only (+, -, *, /, sqrt,
comparisons) on uniform draws from numpy's PCG64 stream, so the same seed
produces bit-identical coordinates on x86-64 and AArch64 hosts.
"""
from __future__ import annotations

import numpy as np

# Element numbers used by the model: H and the sp-basis heavy atoms C, N, O.
H, C, N, O = 1, 6, 7, 8
HEAVY = (C, N, O)
VALENCE_ELECTRONS = {H: 1, C: 4, N: 5, O: 6}
BONDING_VALENCE = {H: 1, C: 4, N: 3, O: 2}

# cos(100 deg) and cos(125 deg), written out so no libm call is involved.
_COS_100 = -0.17364817766693033
_COS_125 = -0.57357643635104605


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _norm(v):
    return np.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])


def _cross(a, b):
    return np.array([a[1] * b[2] - a[2] * b[1],
                     a[2] * b[0] - a[0] * b[2],
                     a[0] * b[1] - a[1] * b[0]])


def _dist2_to(xyz, p):
    dx = xyz[:, 0] - p[0]
    dy = xyz[:, 1] - p[1]
    dz = xyz[:, 2] - p[2]
    return dx * dx + dy * dy + dz * dz


def _unit_disk(rng):
    """Uniform direction in the plane as (c, s) with c^2+s^2=1, by rejection."""
    while True:
        u, v = rng.uniform(-1.0, 1.0, size=2)
        r2 = u * u + v * v
        if 0.01 < r2 <= 1.0:
            r = np.sqrt(r2)
            return u / r, v / r


def _unit_sphere(rng):
    """Uniform direction in space, by rejection from the cube."""
    while True:
        p = rng.uniform(-1.0, 1.0, size=3)
        r2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2]
        if 0.01 < r2 <= 1.0:
            return p / np.sqrt(r2)


def _assign_heteroatoms(n_heavy, n_h, rng):
    """Element list of a saturated chain with n_h hydrogens.

    Starting from all carbon, the bonding valence must drop by
    delta = 4 n - (n_h + 2 (n - 1)).  Each O site lowers it by 2, each N site
    by 1.  The number of sites m is drawn between ceil(delta/2) (all O) and
    min(delta, ceil(n/2)), and the sites are an isolated set along the chain
    (no two heteroatoms bonded), chosen by a left-to-right scan that skips
    positions at random while there is room.  When delta exceeds what isolated
    sites can absorb the remaining steps go to any site (C -> N -> O).
    """
    z = np.full(n_heavy, C, dtype=np.int32)
    delta = 4 * n_heavy - (n_h + 2 * (n_heavy - 1))
    if delta <= 0:
        return z
    cap = (n_heavy + 1) // 2
    lo = (delta + 1) // 2
    hi = min(delta, cap)
    if lo <= hi:
        m = int(rng.integers(lo, hi + 1))
        n_o = delta - m
        sites = []
        k = 0
        while len(sites) < m and k < n_heavy:
            room = ((n_heavy - k) + 1) // 2 - (m - len(sites))   # spare isolated slots from k on
            if room > 0 and rng.uniform() < 0.5:
                k += 1
                continue
            sites.append(k)
            k += 2
        sites = np.array(sites, dtype=np.int64)
        kinds = rng.permutation(len(sites))
        for j, site in enumerate(sites):
            z[site] = O if kinds[j] < n_o else N
        return z
    # too many heteroatoms to keep apart: one valence step at a time anywhere
    total = 4 * n_heavy
    target = total - delta
    while total > target:
        cand = np.nonzero(z != O)[0]
        if cand.size == 0:
            break
        k = int(cand[int(rng.integers(0, cand.size))])
        z[k] = N if z[k] == C else O
        total -= 1
    return z


def _substituent_directions(bonds, count, rng):
    """Unit vectors for ``count`` substituents around an atom whose existing
    bonds point along the unit vectors in ``bonds`` (0, 1 or 2 of them),
    in tetrahedral directions (cos = -1/3 between substituents)."""
    c_t = 0.33333333333333331        # |cos(109.47 deg)|
    s_t = 0.94280904158206336        # sin(109.47 deg)
    if len(bonds) == 0:
        b = _unit_sphere(rng)
        return ([b] + _substituent_directions([b], count - 1, rng))[:count]
    if len(bonds) == 1:
        b = bonds[0]
        ref = np.array([0.0, 0.0, 1.0]) if abs(b[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
        e1 = _cross(b, ref)
        e1 = e1 / _norm(e1)
        e2 = _cross(b, e1)
        c0, s0 = _unit_disk(rng)
        out = []
        # three directions at 120 degree steps around -b
        rot = [(1.0, 0.0), (-0.5, 0.86602540378443860), (-0.5, -0.86602540378443860)]
        for cr, sr in rot[:count]:
            cph = c0 * cr - s0 * sr
            sph = s0 * cr + c0 * sr
            out.append(-c_t * b + s_t * (cph * e1 + sph * e2))
        return out
    b1, b2 = bonds[0], bonds[1]
    m = -(b1 + b2)
    m = m / _norm(m)
    nrm = _cross(b1, b2)
    nn = _norm(nrm)
    if nn < 1e-8:
        ref = np.array([0.0, 0.0, 1.0]) if abs(b1[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
        nrm = _cross(b1, ref)
        nn = _norm(nrm)
    nrm = nrm / nn
    if count == 1:
        return [m]
    # half the tetrahedral angle: cos(54.74 deg), sin(54.74 deg)
    ch, sh = 0.57735026918962584, 0.81649658092772603
    return [ch * m + sh * nrm, ch * m - sh * nrm][:count]


def make_chain(seed: int, n_heavy: int, n_h: int, *,
               bond=(1.0, 1.5), h_bond=(1.0, 1.1), heavy_clash=2.5, h_clash=1.6,
               min_pair=0.9):
    """Seeded saturated heavy-atom chain with attached hydrogens.

    Heavy atoms follow a self-avoiding random walk: bond length U[bond],
    interior bond angle with cosine uniform between cos(125 deg) and
    cos(100 deg), dihedral uniform, non-neighbouring heavy atoms at least
    ``heavy_clash`` apart.  The elements make the chain saturated with
    exactly n_h hydrogens (bonding valence C 4, N 3, O 2), heteroatoms kept
    apart from each other (see _assign_heteroatoms), so the molecule is
    closed shell.  Hydrogens sit at U[h_bond]
    Angstrom in tetrahedral directions around their parent (random phase for
    chain ends), nudged at random while closer than ``h_clash`` to any other
    atom.  Only when n_h exceeds what all-carbon saturation holds are the
    extra hydrogens put round-robin on the heavy atoms.

    Returns (Z, xyz): int32 element numbers and float64 coordinates in
    Angstrom, heavy atoms first in chain order, then hydrogens.
    """
    rng = _rng(seed)
    n_heavy = int(n_heavy)
    n_h = int(n_h)
    if n_heavy < 1:
        raise ValueError("need at least one heavy atom")
    z_heavy = _assign_heteroatoms(n_heavy, n_h, rng)

    pos = np.zeros((n_heavy, 3))
    if n_heavy > 1:
        pos[1] = [rng.uniform(*bond), 0.0, 0.0]
    k = 2
    attempts = 0
    stuck = 0
    while k < n_heavy:
        attempts += 1
        if attempts > 2000 * n_heavy:
            raise RuntimeError("chain walk failed to place atoms")
        if stuck > 200 and k > 3:
            # dead end of the self-avoiding walk: step back and regrow
            k -= 2
            stuck = 0
            continue
        b = pos[k - 1] - pos[k - 2]
        b = b / _norm(b)
        ref = np.array([0.0, 0.0, 1.0]) if abs(b[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
        e1 = _cross(b, ref)
        e1 = e1 / _norm(e1)
        e2 = _cross(b, e1)
        cth = rng.uniform(_COS_125, _COS_100)
        sth = np.sqrt(1.0 - cth * cth)
        cph, sph = _unit_disk(rng)
        length = rng.uniform(*bond)
        # the interior angle at atom k-1 has cosine (-b).d = cth
        d = -cth * b + sth * (cph * e1 + sph * e2)
        p = pos[k - 1] + length * d
        if k >= 3:
            d2 = _dist2_to(pos[: k - 2], p)   # atom k-2 is the 1-3 neighbour
            if np.min(d2) < heavy_clash * heavy_clash:
                stuck += 1
                continue
        pos[k] = p
        k += 1
        stuck = 0

    degree = np.zeros(n_heavy, dtype=np.int64)
    if n_heavy > 1:
        degree[0] += 1
        degree[-1] += 1
        degree[1:-1] += 2
    free = np.array([max(BONDING_VALENCE[int(z)] - int(dg), 0) for z, dg in zip(z_heavy, degree)])
    count = free.copy()
    extra = n_h - int(count.sum())
    j = 0
    while extra > 0:                      # only when all-carbon saturation is exceeded
        count[j % n_heavy] += 1
        extra -= 1
        j += 1
    while extra < 0:                      # only if balancing could not reach the target
        cand = np.nonzero(count > 0)[0]
        count[cand[j % cand.size]] -= 1
        extra += 1
        j += 1

    xyz = [p for p in pos]
    for a in range(n_heavy):
        if count[a] == 0:
            continue
        bonds = []
        for nb in (a - 1, a + 1):
            if 0 <= nb < n_heavy:
                v = pos[nb] - pos[a]
                bonds.append(v / _norm(v))
        ideal = _substituent_directions(bonds, min(int(count[a]), 4 - len(bonds)), rng)
        while len(ideal) < count[a]:
            ideal.append(_unit_sphere(rng))
        for d0 in ideal:
            length = rng.uniform(*h_bond)
            best = None
            for trial in range(300):
                if trial == 0:
                    d = d0
                else:
                    jitter = 0.15 + 0.6 * trial / 300.0
                    d = d0 + jitter * _unit_sphere(rng)
                    d = d / _norm(d)
                p = pos[a] + length * d
                d2 = _dist2_to(np.array(xyz), p)
                d2[a] = np.inf
                m2 = np.min(d2)
                if best is None or m2 > best[0]:
                    best = (m2, p)
                if m2 >= h_clash * h_clash:
                    break
            xyz.append(best[1])

    Z = np.concatenate([z_heavy, np.full(n_h, H, dtype=np.int32)])
    xyz = np.array(xyz, dtype=np.float64)
    nel = sum(VALENCE_ELECTRONS[int(z)] for z in Z)
    if nel % 2 == 1:
        idx_n = np.nonzero(Z == N)[0]
        idx_c = np.nonzero(Z == C)[0]
        if idx_n.size:
            Z[idx_n[0]] = C
        elif idx_c.size:
            Z[idx_c[0]] = N
        else:
            raise RuntimeError("cannot fix electron parity")
    for i in range(len(Z)):
        d2 = _dist2_to(xyz[i + 1:], xyz[i])
        if d2.size and np.min(d2) < min_pair * min_pair:
            raise RuntimeError("atoms closer than the minimum pair distance")
    return Z.astype(np.int32), xyz


# Parameter ranges (eV, Angstrom, 1/Angstrom).  These are physical ranges,
# not the AM1 values, which the paper does not print.
_RANGES_HEAVY = {
    C: dict(Uss=(-55.0, -45.0), Upp=(-42.0, -35.0)),
    N: dict(Uss=(-75.0, -65.0), Upp=(-65.0, -55.0)),
    O: dict(Uss=(-100.0, -90.0), Upp=(-85.0, -75.0)),
}

PARAM_FIELDS = ("Uss", "Upp", "beta_s", "beta_p", "gss", "gsp", "gpp", "gp2", "hsp",
                "D1", "D2", "zeta_s", "zeta_p")


def make_params(seed: int):
    """Seeded per-element synthetic NDDO parameter set for H, C, N, O.

    Returns a dict Z -> dict(field -> float) with the fields of PARAM_FIELDS.
    The one-centre block over (ss, pxpx, pypy, pzpz) is drawn positive
    definite (gp2 < gpp and 3 gsp^2 < 0.95 gss (gpp + 2 gp2)).
    """
    rng = _rng(seed)
    out = {}
    for z in (H, C, N, O):
        p = {}
        if z == H:
            p["Uss"] = rng.uniform(-13.0, -11.0)
            p["Upp"] = 0.0
            p["beta_s"] = rng.uniform(-14.0, -9.0)
            p["beta_p"] = 0.0
            p["gss"] = rng.uniform(11.0, 14.0)
            p["gsp"] = p["gpp"] = p["gp2"] = p["hsp"] = 0.0
            p["D1"] = p["D2"] = 0.0
            p["zeta_s"] = rng.uniform(1.1, 1.4)
            p["zeta_p"] = 0.0
        else:
            r = _RANGES_HEAVY[z]
            p["Uss"] = rng.uniform(*r["Uss"])
            p["Upp"] = rng.uniform(*r["Upp"])
            p["beta_s"] = rng.uniform(-32.0, -21.0)
            p["beta_p"] = rng.uniform(-30.0, -16.0)
            p["gss"] = rng.uniform(10.0, 17.0)
            p["gpp"] = rng.uniform(9.0, 16.0)
            p["gp2"] = rng.uniform(8.0, min(14.0, p["gpp"] - 0.5))
            gsp_max = min(16.0, np.sqrt(0.95 * p["gss"] * (p["gpp"] + 2.0 * p["gp2"]) / 3.0))
            p["gsp"] = rng.uniform(min(9.0, 0.8 * gsp_max), gsp_max)
            p["hsp"] = rng.uniform(0.5, 3.0)
            p["D1"] = rng.uniform(0.3, 0.8)
            p["D2"] = rng.uniform(0.3, 0.7)
            p["zeta_s"] = rng.uniform(1.0, 1.4)
            p["zeta_p"] = rng.uniform(1.0, 1.5)
        out[z] = p
    return out


def params_table(params) -> np.ndarray:
    """Parameters as a dense float64 table [4 elements (H, C, N, O)] x PARAM_FIELDS."""
    return np.array([[params[z][f] for f in PARAM_FIELDS] for z in (H, C, N, O)], dtype=np.float64)


def n_orbitals(Z) -> int:
    return int(sum(4 if int(z) != H else 1 for z in Z))


def n_occupied(Z) -> int:
    nel = sum(VALENCE_ELECTRONS[int(z)] for z in Z)
    if nel % 2:
        raise ValueError("odd electron count: closed shell only")
    return nel // 2


def trial_vectors(seed: int, nvec: int, nocc: int, nvir: int) -> np.ndarray:
    """Seeded trial amplitudes, shape (nvec, nocc, nvir), uniform in [-1, 1)."""
    rng = _rng(seed)
    return rng.uniform(-1.0, 1.0, size=(nvec, nocc, nvir))


def orthonormal_matrix(seed: int, n: int) -> np.ndarray:
    """A seeded n x n orthonormal matrix (QR of a uniform matrix, signs fixed)."""
    rng = _rng(seed)
    a = rng.uniform(-1.0, 1.0, size=(n, n))
    q, r = np.linalg.qr(a)
    return q * np.sign(np.diag(r))[None, :]


# ---- the workloads of the paper's benchmarks, as seeded stand-ins -------------

def config_small(seed: int = 0):
    """12 heavy atoms + 14 H, 62 AOs (CIS, 5 roots, brute-force checkable)."""
    return make_chain(seed, 12, 14)


def config_medium(seed: int = 0):
    """100 heavy atoms + 200 H, 600 AOs (CIS and TDHF, 10 roots)."""
    return make_chain(seed, 100, 200)


def config_large(seed: int = 0):
    """400 heavy atoms + 600 H, 2200 AOs (TDHF, 10 roots)."""
    return make_chain(seed, 400, 600)


def config_batch(seed: int):
    """One molecule of the batched set: N ~ U{20..200} atoms, 40% heavy."""
    rng = _rng(10_000_000 + int(seed))
    n_atoms = int(rng.integers(20, 201))
    n_heavy = max(1, int(round(0.4 * n_atoms)))
    return make_chain(seed, n_heavy, n_atoms - n_heavy)


def config_sized(seed: int, n_atoms: int, heavy_frac: float = 0.4):
    n_heavy = max(1, int(round(heavy_frac * n_atoms)))
    return make_chain(seed, n_heavy, n_atoms - n_heavy)
