"""Seeded synthetic inputs: tetrahedral meshes, reaction-diffusion models and
initial molecule placements shaped like the workloads of Parallel STEPS (§3).

This module is shared by the CUDA path, the CPU oracle and the tests. It holds
none of the method's arithmetic: no volumes, areas, rates, time windows or
sampling of the simulation itself. It only builds vertex/tet arrays, model
tables in SI units and integer molecule counts from numpy's seeded generators.

Units: vertex coordinates in metres, diffusion constants in m^2/s, rate
constants in SI (order 0: M/s, order 1: 1/s, order 2: 1/(M s)).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import permutations

import numpy as np

UM = 1e-6  # one micrometre in metres


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def kuhn_box_mesh(nx: int, ny: int, nz: int, h: float, origin=(0.0, 0.0, 0.0)):
    """Cube grid of nx*ny*nz cubes of edge h, each split into the 6 Kuhn tets
    that share the cube's main diagonal. Every cube uses the same split, so
    neighbouring cubes meet on matching triangles (a conforming mesh).

    Tet order: cube-major (x fastest), 6 tets per cube. Returns
    (verts [nv,3] float64, tets [nt,4] int32)."""
    gx, gy, gz = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    verts = np.stack([gx.ravel(order="F"), gy.ravel(order="F"), gz.ravel(order="F")], axis=1).astype(np.float64)
    verts = verts * h + np.asarray(origin, dtype=np.float64)

    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(order="F"), cj.ravel(order="F"), ck.ravel(order="F")
    unit = np.eye(3, dtype=np.int64)
    tets = []
    for perm in permutations(range(3)):
        a, b = unit[perm[0]], unit[perm[1]]
        ab = a + b
        t = np.stack([
            vid(ci, cj, ck),
            vid(ci + a[0], cj + a[1], ck + a[2]),
            vid(ci + ab[0], cj + ab[1], ck + ab[2]),
            vid(ci + 1, cj + 1, ck + 1),
        ], axis=1)
        tets.append(t)
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return verts, tets


def jitter_box_vertices(verts: np.ndarray, h: float, frac: float, seed: int):
    """Move every vertex by an independent uniform offset in [-frac*h, frac*h]
    per axis, except along axes where it lies on the box boundary (a vertex on a
    face moves within that face, an edge vertex along its edge, corners stay).
    The box surface, and so the total volume, is unchanged. For frac <= 0.2 a
    Kuhn tet cannot invert: its smallest altitude is h/sqrt(2) ~ 0.71h while the
    displacement normal to any face plane is at most 2*frac*h*sqrt(2) ~ 0.57h."""
    rng = np.random.default_rng(seed)
    lo = verts.min(axis=0)
    hi = verts.max(axis=0)
    tol = 1e-9 * h
    free = (np.abs(verts - lo) > tol) & (np.abs(verts - hi) > tol)
    off = rng.uniform(-frac * h, frac * h, size=verts.shape)
    return verts + np.where(free, off, 0.0)


def isolated_tets(n: int, edge: float = 0.5 * UM, spacing: float = 1.0 * UM):
    """n disjoint copies of one Kuhn tet of a cube of edge `edge`, laid out on
    a line: no two share a face, so each is an independent well-mixed
    compartment (one tet = one replicate)."""
    base = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1]], dtype=np.float64) * edge
    shift = np.zeros((n, 1, 3))
    shift[:, 0, 0] = np.arange(n) * spacing
    verts = (base[None] + shift).reshape(-1, 3)
    tets = np.arange(4 * n, dtype=np.int32).reshape(n, 4)
    return verts, tets


def isolated_pairs(n: int, edge: float = 0.5 * UM, spacing: float = 2.0 * UM):
    """n disjoint pairs of face-sharing tets (two Kuhn tets of one cube):
    n independent 2-tet meshes in one mesh."""
    base = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1], [0, 1, 0]], dtype=np.float64) * edge
    # tet 0: (v0, v1, v2, v3) = x-then-y path; tet 1: (v0, v4, v2, v3) = y-then-x path;
    # they share the face (v0, v2, v3).
    shift = np.zeros((n, 1, 3))
    shift[:, 0, 0] = np.arange(n) * spacing
    verts = (base[None] + shift).reshape(-1, 3)
    off = (5 * np.arange(n, dtype=np.int64))[:, None]
    t0 = np.array([0, 1, 2, 3])[None] + off
    t1 = np.array([0, 4, 2, 3])[None] + off
    tets = np.stack([t0, t1], axis=1).reshape(-1, 4).astype(np.int32)
    return verts, tets


@dataclass
class _Segment:
    p0: np.ndarray
    p1: np.ndarray
    r: float


def _branch_tree(seed: int, levels: int, root_r: float, root_len: float):
    """Binary tree of cylinders: each level's radius is 0.6x and length 0.8x
    its parent's, branching angles drawn in [30, 60] degrees."""
    rng = np.random.default_rng(seed)
    segs = []

    def grow(p0, direction, r, length, level):
        p1 = p0 + direction * length
        segs.append(_Segment(p0, p1, r))
        if level + 1 >= levels:
            return
        for side in (-1.0, 1.0):
            ang = np.deg2rad(rng.uniform(30.0, 60.0)) * side
            # rotate in a plane spanned by `direction` and a random normal
            n = rng.normal(size=3)
            n -= n.dot(direction) * direction
            n /= np.linalg.norm(n)
            d = np.cos(ang) * direction + np.sin(ang) * n
            d /= np.linalg.norm(d)
            grow(p1, d, r * 0.6, length * 0.8, level + 1)

    grow(np.zeros(3), np.array([1.0, 0.0, 0.0]), root_r, root_len, 0)
    return segs


def dendrite_mesh(seed: int = 1, h: float = 0.149 * UM, levels: int = 5,
                  root_r: float = 2.0 * UM, root_len: float = 20.0 * UM):
    """Branching dendrite: a binary tree of capsules voxelised on a cubic grid
    of edge h (a cube is kept when its centre lies inside any capsule), each
    kept cube split into 6 Kuhn tets sharing the grid's vertices, so the mesh
    is conforming. Returns (verts, tets, soma_axis_coord) where the last value
    is each tet's cube-centre coordinate along the root axis (used to mark the
    soma end)."""
    segs = _branch_tree(seed, levels, root_r, root_len)
    pts = np.concatenate([np.stack([s.p0, s.p1]) for s in segs])
    rmax = max(s.r for s in segs)
    lo = pts.min(axis=0) - rmax - h
    hi = pts.max(axis=0) + rmax + h
    n = np.ceil((hi - lo) / h).astype(np.int64)
    occ = np.zeros(n, dtype=bool)
    for s in segs:
        slo = np.floor((np.minimum(s.p0, s.p1) - s.r - lo) / h).astype(np.int64)
        shi = np.ceil((np.maximum(s.p0, s.p1) + s.r - lo) / h).astype(np.int64)
        slo = np.clip(slo, 0, n)
        shi = np.clip(shi, 0, n)
        ix = np.arange(slo[0], shi[0])
        iy = np.arange(slo[1], shi[1])
        iz = np.arange(slo[2], shi[2])
        cx, cy, cz = np.meshgrid(ix, iy, iz, indexing="ij")
        c = np.stack([cx, cy, cz], axis=-1).reshape(-1, 3)
        x = lo + (c + 0.5) * h
        d = s.p1 - s.p0
        t = np.clip(((x - s.p0) @ d) / d.dot(d), 0.0, 1.0)
        dist = np.linalg.norm(x - (s.p0 + t[:, None] * d), axis=1)
        inside = c[dist <= s.r]
        occ[inside[:, 0], inside[:, 1], inside[:, 2]] = True
    cubes = np.argwhere(occ)  # row-major (x slowest); keep for locality below
    order = np.lexsort((cubes[:, 0], cubes[:, 1], cubes[:, 2]))
    cubes = cubes[order]
    # vertex ids on the (n+1)^3 lattice, compacted to the used ones
    def lat(i, j, k):
        return i + (n[0] + 1) * (j + (n[1] + 1) * k)

    unit = np.eye(3, dtype=np.int64)
    ci, cj, ck = cubes[:, 0], cubes[:, 1], cubes[:, 2]
    tl = []
    for perm in permutations(range(3)):
        a, b = unit[perm[0]], unit[perm[1]]
        ab = a + b
        tl.append(np.stack([
            lat(ci, cj, ck),
            lat(ci + a[0], cj + a[1], ck + a[2]),
            lat(ci + ab[0], cj + ab[1], ck + ab[2]),
            lat(ci + 1, cj + 1, ck + 1),
        ], axis=1))
    tl = np.stack(tl, axis=1).reshape(-1, 4)
    used, inv = np.unique(tl.ravel(), return_inverse=True)
    tets = inv.reshape(-1, 4).astype(np.int32)
    k_ = used // ((n[0] + 1) * (n[1] + 1))
    rem = used % ((n[0] + 1) * (n[1] + 1))
    j_ = rem // (n[0] + 1)
    i_ = rem % (n[0] + 1)
    verts = lo + np.stack([i_, j_, k_], axis=1).astype(np.float64) * h
    axis_coord = np.repeat(lo[0] + (ci + 0.5) * h, 6)
    return verts, tets, axis_coord


# --------------------------------------------------------------------------
# models
# --------------------------------------------------------------------------

@dataclass
class Model:
    """Species and reactions in SI units.

    lhs/rhs are [R, S] stoichiometry matrices (reactant and product molecule
    counts); k[r] is the macroscopic rate constant of reaction r."""
    names: list
    diff: np.ndarray  # [S] m^2/s, 0 = immobile
    lhs: np.ndarray  # [R, S] int32
    rhs: np.ndarray  # [R, S] int32
    k: np.ndarray  # [R] float64
    reac_names: list = field(default_factory=list)

    @property
    def n_species(self):
        return len(self.names)

    @property
    def n_reac(self):
        return self.lhs.shape[0]


def _model(names, diff, reactions):
    s_idx = {n: i for i, n in enumerate(names)}
    S, R = len(names), len(reactions)
    lhs = np.zeros((R, S), np.int32)
    rhs = np.zeros((R, S), np.int32)
    k = np.zeros(R)
    rn = []
    for r, (left, right, rate) in enumerate(reactions):
        for n in left:
            lhs[r, s_idx[n]] += 1
        for n in right:
            rhs[r, s_idx[n]] += 1
        k[r] = rate
        rn.append(" + ".join(left) + " -> " + " + ".join(right))
    return Model(list(names), np.asarray(diff, dtype=np.float64), lhs, rhs, k, rn)


def model_from_lists(names, diff, reactions):
    """Model from species names, D per species and a list of
    (reactant names, product names, k) tuples."""
    return _model(names, diff, reactions)


def config1_model():
    """A + B <-> C, kf = 1e6 /M/s, kb = 10 /s, D = 1e-11 m^2/s for all."""
    return _model(["A", "B", "C"], [1e-11, 1e-11, 1e-11],
                  [(["A", "B"], ["C"], 1e6), (["C"], ["A", "B"], 10.0)])


def random_network(seed: int, n_species: int = 10, n_first: int = 10, n_second: int = 10,
                   d_range=(1e-13, 1e-11), k1_range=(1e-1, 1e3), k2_range=(1e5, 1e8)):
    """Random network: first-order conversions X -> Y and dissociations
    Z -> X + Y, second-order bindings X + Y -> Z (X != Y, no homodimers);
    rates and D log-uniform."""
    rng = np.random.default_rng(seed)
    names = [f"S{i}" for i in range(n_species)]

    def logu(lo, hi, size=None):
        return np.exp(rng.uniform(np.log(lo), np.log(hi), size=size))

    diff = logu(*d_range, size=n_species)
    reactions = []
    for r in range(n_first):
        if r % 2 == 0:
            x, y = rng.choice(n_species, 2, replace=False)
            reactions.append(([names[x]], [names[y]], float(logu(*k1_range))))
        else:
            z, x, y = rng.choice(n_species, 3, replace=False)
            reactions.append(([names[z]], [names[x], names[y]], float(logu(*k1_range))))
    for r in range(n_second):
        x, y, z = rng.choice(n_species, 3, replace=False)
        reactions.append(([names[x], names[y]], [names[z]], float(logu(*k2_range))))
    return _model(names, diff, reactions)


def calcium_model(d_ca: float = 2e-10, seed: int = 7):
    """Calcium-buffering network with 20 species: Ca; four two-site buffers
    (B, CaB, Ca2B each); seven inert diffusive tracers. Reactions: sequential
    Ca binding/unbinding on each buffer (16), a first-order pump Ca -> 0 and a
    zero-order influx 0 -> Ca (to be masked to the soma end)."""
    rng = np.random.default_rng(seed)
    names = ["Ca"]
    diff = [d_ca]
    reactions = []
    buf_d = [1e-11, 1e-12, 1e-13, 0.0]
    for b in range(4):
        B, CB, C2B = f"B{b}", f"CaB{b}", f"Ca2B{b}"
        names += [B, CB, C2B]
        diff += [buf_d[b]] * 3
        kon = float(np.exp(rng.uniform(np.log(1e7), np.log(5e8))))
        koff = float(np.exp(rng.uniform(np.log(1e1), np.log(1e3))))
        reactions += [(["Ca", B], [CB], kon), ([CB], ["Ca", B], koff),
                      (["Ca", CB], [C2B], kon * 0.5), ([C2B], ["Ca", CB], koff * 2.0)]
    for t in range(7):
        names.append(f"T{t}")
        diff.append(float(np.exp(rng.uniform(np.log(1e-12), np.log(1e-11)))))
    reactions.append((["Ca"], [], 1e3))          # pump
    reactions.append(([], ["Ca"], 5e-3))          # influx (M/s), masked region
    return _model(names, diff, reactions)


# --------------------------------------------------------------------------
# placement
# --------------------------------------------------------------------------

def place_uniform(total: int, n_tets: int, seed: int, subset=None):
    """Per-tet counts for `total` molecules, each placed independently in a tet
    drawn uniformly from `subset` (default: all tets). On the meshes here all
    tets of one grid have the same nominal volume, so this matches placement by
    volume up to the jitter."""
    rng = np.random.default_rng(seed)
    out = np.zeros(n_tets, dtype=np.int32)
    idx = np.arange(n_tets) if subset is None else np.asarray(subset)
    if total > 0 and len(idx) > 0:
        cnt = rng.multinomial(total, np.full(len(idx), 1.0 / len(idx)))
        out[idx] = cnt.astype(np.int32)
    return out


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    verts: np.ndarray
    tets: np.ndarray
    model: Model
    counts: np.ndarray  # [S, nt] int32, original tet order
    t_end: float
    seed: int
    reac_masks: dict = field(default_factory=dict)  # r -> uint8 [nt]

    @property
    def n_tets(self):
        return self.tets.shape[0]


def config1(seed: int = 3):
    """2x2x10 um cuboid, 4x4x20 cubes of 0.5 um -> 1920 tets; A + B <-> C;
    5000 A and 5000 B placed uniformly; 10 ms."""
    verts, tets = kuhn_box_mesh(4, 4, 20, 0.5 * UM)
    m = config1_model()
    nt = tets.shape[0]
    counts = np.zeros((3, nt), np.int32)
    counts[0] = place_uniform(5000, nt, seed=2)
    counts[1] = place_uniform(5000, nt, seed=12)
    return Workload("cuboid-1920tets-A+B<->C-10ms", verts, tets, m, counts, 10e-3, seed)


def config2(seed: int = 3, nx: int = 170, ny: int = 17, nz: int = 17, t_end: float = 20e-3,
            net_seed: int = 5, h: float = None, density_scale: float = 1.0):
    """100x10x10 um box of 170x17x17 cubes (h = 10/17 um) x 6 tets = 294,780
    tets, vertices jittered by 20% of the spacing; random 10-species,
    20-reaction network; densities U[1, 100] /um^3 per species (times
    density_scale); 20 ms. h sets another cube edge (the mesh-coarseness
    experiment: the same box with nx = 10 n, ny = nz = n, h = 10/n um)."""
    h = 10.0 / 17.0 * UM if h is None else h
    verts, tets = kuhn_box_mesh(nx, ny, nz, h)
    verts = jitter_box_vertices(verts, h, 0.2, seed=1)
    m = random_network(net_seed)
    nt = tets.shape[0]
    rng = np.random.default_rng(2)
    vol_um3 = nx * ny * nz * (h / UM) ** 3
    dens = rng.uniform(1.0, 100.0, size=m.n_species) * density_scale
    counts = np.zeros((m.n_species, nt), np.int32)
    for s in range(m.n_species):
        counts[s] = place_uniform(int(round(dens[s] * vol_um3)), nt, seed=100 + s)
    return Workload(f"irregular-box-{nt}tets-10sp-20rx-{t_end*1e3:g}ms", verts, tets, m, counts, t_end, seed)


def config3(seed: int = 3, h: float = 0.149 * UM, t_end: float = 50e-3):
    """Dendrite tree (5 levels, root r = 2 um, L = 20 um) voxelised to ~1M tets;
    20-species calcium-buffering network; Ca placed in the soma-end 5% of tets;
    influx masked to the same tets; 50 ms."""
    verts, tets, axis = dendrite_mesh(seed=1, h=h)
    m = calcium_model()
    nt = tets.shape[0]
    soma = np.argsort(axis, kind="stable")[: max(1, nt // 20)]
    vol_um3 = nt / 6 * (h / UM) ** 3
    counts = np.zeros((m.n_species, nt), np.int32)
    rng = np.random.default_rng(2)
    for s, name in enumerate(m.names):
        if name == "Ca":
            counts[s] = place_uniform(int(round(50.0 * vol_um3)), nt, seed=200, subset=soma)
        elif name.startswith("B"):
            counts[s] = place_uniform(int(round(rng.uniform(20, 60) * vol_um3)), nt, seed=200 + s)
        elif name.startswith("T"):
            counts[s] = place_uniform(int(round(rng.uniform(1, 10) * vol_um3)), nt, seed=200 + s)
    mask = np.zeros(nt, np.uint8)
    mask[soma] = 1
    influx = m.n_reac - 1
    return Workload(f"dendrite-{nt}tets-20sp-{m.n_reac}rx-{t_end*1e3:g}ms", verts, tets, m, counts,
                    t_end, seed, reac_masks={influx: mask})


def batch_sizes(n: int = 256, lo: int = 10_000, hi: int = 300_000, seed: int = 11):
    """Tet counts log-uniform in [lo, hi] for n replicates."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))


def box_for_tets(target: int, seed: int, t_end: float = 20e-3, net_seed: int = 5):
    """A config-2-style jittered box with about `target` tets (cross-section
    17x17 cubes, length chosen to match), same network generator."""
    nx = max(1, int(round(target / (6 * 17 * 17))))
    return config2(seed=seed, nx=nx, t_end=t_end, net_seed=net_seed)


def replicate_mesh(verts: np.ndarray, tets: np.ndarray, n: int, spacing: float):
    """n disjoint copies of one mesh, shifted along x by `spacing` each (must
    exceed the mesh's x extent): copy c owns tets [c*nt, (c+1)*nt)."""
    nv = verts.shape[0]
    shift = np.zeros((n, 1, 3))
    shift[:, 0, 0] = np.arange(n) * spacing
    v = (verts[None] + shift).reshape(-1, 3)
    t = (tets[None].astype(np.int64) + (np.arange(n) * nv)[:, None, None]).reshape(-1, 4)
    return v, t.astype(np.int32)


# --------------------------------------------------------------------------
# served job stream
# --------------------------------------------------------------------------

SIZE_BUCKETS = np.unique(np.round(np.geomspace(2_000, 1_000_000, 10)).astype(np.int64))


def bucket_of(n_tets: int) -> int:
    """Nearest size bucket (log scale) for a requested tet count."""
    i = int(np.argmin(np.abs(np.log(SIZE_BUCKETS) - np.log(max(n_tets, 1)))))
    return int(SIZE_BUCKETS[i])


def config1_scaled(target: int, seed: int = 3, t_end: float = 10e-3):
    """Config-1 chemistry (A + B <-> C) on a 4x4xL grid of 0.5 um cubes sized
    to about `target` tets, 125 A and 125 B per um^3."""
    L = max(1, int(round(target / 96)))
    verts, tets = kuhn_box_mesh(4, 4, L, 0.5 * UM)
    m = config1_model()
    nt = tets.shape[0]
    n = int(round(125.0 * 2 * 2 * L * 0.5))
    counts = np.zeros((3, nt), np.int32)
    counts[0] = place_uniform(n, nt, seed=2)
    counts[1] = place_uniform(n, nt, seed=12)
    return Workload(f"cuboid-{nt}tets-A+B<->C", verts, tets, m, counts, t_end, seed)


def config3_scaled(target: int, seed: int = 3, t_end: float = 50e-3):
    """Config-3 dendrite and calcium network, voxel edge chosen so that the
    mesh has about `target` tets (0.149 um gives ~1.03M)."""
    h = 0.149 * UM * (1.03e6 / max(target, 1)) ** (1.0 / 3.0)
    return config3(seed=seed, h=h, t_end=t_end)


def make_job_workload(kind: int, size: int, seed: int, t_end: float):
    """Workload of a served job: generator `kind` (1, 2 or 3) scaled to about
    `size` tets."""
    if kind == 1:
        w = config1_scaled(size, seed=seed, t_end=t_end)
    elif kind == 2:
        w = box_for_tets(size, seed=seed, t_end=t_end)
    else:
        w = config3_scaled(size, seed=seed, t_end=t_end)
    w.t_end = t_end
    w.seed = seed
    return w


@dataclass
class JobSpec:
    job_id: int
    arrival: float   # seconds after the stream starts
    kind: int        # generator 1, 2 or 3
    size: int        # size bucket (tets, approximate)
    seed: int
    t_end: float     # simulated seconds


def served_jobs(n: int, rate: float = 50.0, seed: int = 21, t_range=(1e-3, 100e-3),
                size_range=(2_000, 1_000_000)):
    """Poisson arrival stream (mean `rate` jobs/s) of n jobs; generator uniform
    over configs 1-3, size log-uniform in size_range (snapped to a bucket),
    t_end log-uniform in t_range, distinct seeds."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    t -= t[0]
    jobs = []
    for j in range(n):
        size = float(np.exp(rng.uniform(np.log(size_range[0]), np.log(size_range[1]))))
        t_end = float(np.exp(rng.uniform(np.log(t_range[0]), np.log(t_range[1]))))
        jobs.append(JobSpec(j, float(t[j]), int(rng.integers(1, 4)), bucket_of(int(size)), 5000 + j, t_end))
    return jobs
