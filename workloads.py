"""Seeded synthetic workloads for the enriched-FE ChFSI path.

This module holds NO arithmetic of the method: it only draws geometry, mesh
break points, enrichment parameters, potential parameters and initial vectors
from seeded NumPy generators (PCG64).  It is the one module shared by the CPU
oracle (``oracle/``) and the CUDA library's Python binding; both sides build
their own operators from these plain descriptions.

Systems follow the shapes of the paper's workloads (Sec. VI): a hydrogen-like
single nucleus (closed-form spectrum), a harmonic oscillator (classical basis
only), and silicon-like diamond-lattice clusters (lattice constant 10.26 bohr,
Sec. VI.B.1) whose real atomic enrichment data are replaced by analytic Slater
radials with seeded exponents.
"""
import math
import numpy as np

A_SI = 10.26  # diamond lattice constant of the paper's silicon clusters (bohr)


def _uniform_breaks(lo, hi, n):
    return np.linspace(lo, hi, n + 1)


def graded_breaks(lo, hi, must, h_min, h_max, growth=1.3, fine_pad=2.0):
    """Per-axis cell break points: every coordinate in ``must`` is a break point,
    cells no longer than ``h_min`` between the first and last of them and within
    ``fine_pad`` of them, then geometric growth (x ``growth``) up to ``h_max``
    towards the box faces.  Pure mesh generation (input structure)."""
    must = np.unique(np.round(np.asarray(must, dtype=np.float64), 12))
    inner = [must[0]]
    for a, b in zip(must[:-1], must[1:]):
        k = max(1, int(math.ceil((b - a) / h_min - 1e-9)))
        inner.extend(list(a + (b - a) * np.arange(1, k + 1) / k))
    inner = np.array(inner)

    def outward(start, end):
        # segments from start towards end (end may be < start)
        sgn = 1.0 if end > start else -1.0
        dist = abs(end - start)
        lens = []
        pad_cells = max(1, int(math.ceil(fine_pad / h_min - 1e-9)))
        for _ in range(pad_cells):
            lens.append(min(h_min, fine_pad / pad_cells))
        h = lens[-1]
        while sum(lens) < dist:
            h = min(h * growth, h_max)
            lens.append(h)
        lens = np.array(lens)
        # shrink the coarse tail so the segments end exactly at the face
        excess = lens.sum() - dist
        if excess > 0:
            if excess > 0.5 * lens[-1] and len(lens) > 1:
                lens = lens[:-1]
                lens[-1] += dist - lens.sum()
            else:
                lens[-1] -= excess
        pts = start + sgn * np.cumsum(lens)
        pts[-1] = end
        return pts

    left = outward(inner[0], lo)[::-1]
    right = outward(inner[-1], hi)
    return np.concatenate([left, inner, right])


def diamond_cluster(nx, ny, nz, a=A_SI):
    """Atoms of nx*ny*nz conventional diamond cells, without boundary duplicates."""
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                      [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])
    pos = []
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                for b in basis:
                    pos.append((np.array([i, j, k]) + b) * a)
    return np.array(pos)


def diamond_cube_cut(ncell, a=A_SI):
    """Cube cut of ncell^3 conventional cells INCLUDING boundary atoms
    (3x3x3 gives the paper's 280-atom cluster, Sec. VI.B.1)."""
    pts = set()
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                      [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])
    for i in range(-1, ncell + 1):
        for j in range(-1, ncell + 1):
            for k in range(-1, ncell + 1):
                for b in basis:
                    f = np.array([i, j, k]) + b
                    if np.all(f >= -1e-9) and np.all(f <= ncell + 1e-9):
                        pts.add(tuple(np.round(f * 4).astype(int)))
    return np.array(sorted(pts), dtype=np.float64) * a / 4.0


def slater_zetas(Z):
    """Slater's-rules exponents (1s, 2s/2p) -- fixed published rules, used only to
    draw plausible synthetic radial exponents."""
    z1 = Z - 0.30 if Z > 1 else 1.0
    if Z <= 2:
        return z1, max(0.5, (Z - 0.85 * (Z - 1)) / 2.0)
    n2 = min(Z - 2, 8)
    s2 = 2 * 0.85 + (n2 - 1) * 0.35
    z2 = (Z - s2) / 2.0
    return z1, z2


def _system(breaks, p, atoms, Z, funcs, potential, n_gauss=6, tau=1e-10,
            max_depth=10, n_adapt=6, name=""):
    return {
        "name": name,
        "p": p,
        "breaks": [np.asarray(b, dtype=np.float64) for b in breaks],
        "n_gauss": n_gauss,
        "atoms": np.asarray(atoms, dtype=np.float64).reshape(-1, 3),
        "Z": np.asarray(Z, dtype=np.float64).reshape(-1),
        "funcs": funcs,
        "potential": potential,
        "quad": {"tau": tau, "max_depth": max_depth, "n": n_adapt},
    }


def _hydrogenic_funcs(atom, r0, t):
    out = []
    for (n, l, m) in [(1, 0, 0), (2, 0, 0), (2, 1, -1), (2, 1, 0), (2, 1, 1)]:
        out.append({"atom": atom, "n": n, "l": l, "m": m, "kind": "hydrogenic",
                    "zeta": 0.0, "r0": r0, "t": t})
    return out


def _slater_funcs(atom, z1, z2, r0, t):
    out = [{"atom": atom, "n": 1, "l": 0, "m": 0, "kind": "slater", "zeta": z1, "r0": r0, "t": t},
           {"atom": atom, "n": 2, "l": 0, "m": 0, "kind": "slater", "zeta": z2, "r0": r0, "t": t}]
    for m in (-1, 0, 1):
        out.append({"atom": atom, "n": 2, "l": 1, "m": m, "kind": "slater", "zeta": z2, "r0": r0, "t": t})
    return out


def hydrogen(cells=6, half=10.0, r_c=6.0, tau=1e-10, max_depth=10, n_gauss=6):
    """Single bare nucleus Z=1 at the centre of a (2*half)^3 box; hydrogenic
    1s,2s,2p enrichment cut off at r_c (r0 = r_c/2, t = 1)."""
    b = _uniform_breaks(-half, half, cells)
    funcs = _hydrogenic_funcs(0, r_c / 2.0, 1.0)
    pot = {"nuclear": True, "gauss_A": np.zeros(0), "gauss_s": np.zeros(0),
           "gauss_c": np.zeros((0, 3)), "omega": 0.0}
    return _system([b, b, b], 4, [[0.0, 0.0, 0.0]], [1.0], funcs, pot, n_gauss=n_gauss,
                   tau=tau, max_depth=max_depth, name=f"hydrogen_{cells}c_{2*half:g}bohr")


def bare_nucleus(Z=14.0, enriched=True, cells=6, half=10.0, r_c=2.0, h_min=None, h_max=3.4, growth=1.3,
                 tau=1e-10, max_depth=12, n_gauss=6):
    """A bare nucleus of charge Z at the centre of a (2 half)^3 box, V = -Z/r: the
    closed-form spectrum -Z^2/(2 n^2) (Z = 14: the Si-like core, 1s at -98 Ha).
    enriched: uniform cells x cells x cells mesh with the hydrogenic 1s, 2s, 2p
    functions of charge Z cut off at r_c (r0 = r_c/2, t = 1); classical
    (n_E = 0): graded mesh refined towards the nucleus down to h_min."""
    if enriched:
        b = _uniform_breaks(-half, half, cells)
        funcs = _hydrogenic_funcs(0, r_c / 2.0, 1.0)
        breaks = [b, b, b]
    else:
        b = graded_breaks(-half, half, [0.0], h_min, h_max, growth=growth, fine_pad=2.0 * h_min)
        funcs = []
        breaks = [b, b, b]
    pot = {"nuclear": True, "gauss_A": np.zeros(0), "gauss_s": np.zeros(0),
           "gauss_c": np.zeros((0, 3)), "omega": 0.0}
    tag = f"enr{cells}" if enriched else f"cls{h_min:g}"
    return _system(breaks, 4, [[0.0, 0.0, 0.0]], [float(Z)], funcs, pot, n_gauss=n_gauss, tau=tau,
                   max_depth=max_depth, name=f"Z{Z:g}_{tag}")


def tiny_heavy(Z=79.0, seed=14, cells=2, half=2.0, r_c=1.6, tau=1e-8, max_depth=8):
    """Heavy nucleus (Z = 79) at the centre vertex of a small uniform mesh with its
    Slater 1s/2s/2p enrichment (Slater's-rules exponents, seeded +-5 %) and a
    seeded Gaussian perturbation: parity case of the heavy-Z stand-in."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = _uniform_breaks(-half, half, cells)
    z1, z2 = slater_zetas(int(Z))
    z1 *= 1.0 + 0.05 * rng.uniform(-1, 1)
    z2 *= 1.0 + 0.05 * rng.uniform(-1, 1)
    funcs = _slater_funcs(0, z1, z2, r_c / 2.0, 1.0)
    pot = {"nuclear": True,
           "gauss_A": rng.uniform(-0.5, 0.5, size=2),
           "gauss_s": rng.uniform(0.5, 1.0, size=2),
           "gauss_c": rng.uniform(-1.0, 1.0, size=(2, 3)),
           "omega": 0.0}
    return _system([b, b, b], 4, [[0.0, 0.0, 0.0]], [float(Z)], funcs, pot, tau=tau, max_depth=max_depth,
                   name=f"heavy{Z:g}")


def gold_dimer(h_min=0.9, h_max=3.0, pad=8.0, r_c=3.0, seed=13, tau=1e-8, max_depth=8):
    """Heavy-Z stand-in (Sec. VI.B.2's gold clusters): two Z = 79 nuclei 4.67 bohr
    apart, graded degree-4 mesh, Slater 1s/2s/2p enrichment per atom (exponents
    from Slater's rules, seeded +-5 %), bare nuclear potential; 158 electrons."""
    atoms = np.array([[0.0, 0.0, 0.0], [4.67, 0.0, 0.0]])
    return _cluster_system(atoms, np.array([79.0, 79.0]), h_min, h_max, pad, r_c, seed, seed + 1, 0, tau, max_depth,
                           name="au2")


def harmonic(cells=8, half=8.0, omega=1.0, p=4):
    """3-D harmonic oscillator V = omega^2 r^2 / 2, classical basis only."""
    b = _uniform_breaks(-half, half, cells)
    pot = {"nuclear": False, "gauss_A": np.zeros(0), "gauss_s": np.zeros(0),
           "gauss_c": np.zeros((0, 3)), "omega": float(omega)}
    return _system([b, b, b], p, np.zeros((0, 3)), np.zeros(0), [], pot,
                   name=f"harmonic_{cells}c")


def tiny(seed=11, cells=(2, 3, 2), n_gauss=6, with_enrichment=True, n_gaussians=3,
         max_depth=4, tau=1e-8):
    """Small non-uniform mesh with two light nuclei and a seeded Gaussian-sum
    potential: brute-force checks and GPU tile / ragged-tail parity cases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    breaks = []
    for n in cells:
        w = rng.uniform(0.7, 1.3, size=n)
        x = np.concatenate([[0.0], np.cumsum(w)])
        x = -4.0 + 8.0 * x / x[-1]
        breaks.append(x)
    # nuclei at interior mesh vertices
    atoms, Z = [], []
    picks = [(1, 1, 1), (1, 2, 1)] if cells[1] >= 3 else [(1, 1, 1)]
    for (i, j, k) in picks:
        atoms.append([breaks[0][i], breaks[1][j], breaks[2][k]])
        Z.append(float(len(Z) + 1))
    funcs = []
    if with_enrichment:
        for ia, z in enumerate(Z):
            if ia == 0:
                funcs += _hydrogenic_funcs(ia, 1.2, 1.0)
            else:
                z1, z2 = slater_zetas(3)
                funcs += _slater_funcs(ia, z1, z2, 1.1, 0.8)[:3]
    pot = {"nuclear": True,
           "gauss_A": rng.uniform(-0.5, 0.5, size=n_gaussians),
           "gauss_s": rng.uniform(0.8, 1.5, size=n_gaussians),
           "gauss_c": rng.uniform(-2.5, 2.5, size=(n_gaussians, 3)),
           "omega": 0.0}
    return _system(breaks, 4, atoms, Z, funcs, pot, n_gauss=n_gauss, tau=tau,
                   max_depth=max_depth, name=f"tiny_s{seed}")


def si_cluster(n_cells_x=2, h_min=0.90, h_max=3.0, pad=10.0, r_c=4.0, seed=2,
               pot_seed=3, n_gaussians=32, tau=1e-9, max_depth=9):
    """16-atom silicon-like cluster (two conventional diamond cells along x,
    Z=14), graded degree-4 mesh, Slater 1s/2s/2p enrichment (5 per atom) with
    exponents from Slater's rules x (1 + 0.05 U(-1,1)), nuclear Coulomb plus a
    seeded 32-term Gaussian perturbation."""
    atoms = diamond_cluster(n_cells_x, 1, 1)
    Z = np.full(len(atoms), 14.0)
    return _cluster_system(atoms, Z, h_min, h_max, pad, r_c, seed, pot_seed, n_gaussians,
                           tau, max_depth, name=f"si{len(atoms)}")


def si280(h_min=1.3, h_max=3.0, pad=10.0, r_c=4.0, seed=4, pot_seed=6, n_gaussians=32, tau=1e-7, max_depth=7):
    """The paper's 280-atom silicon cluster (Sec. VI.B.1): a cube cut of 3 x 3 x 3
    conventional diamond cells including the boundary atoms (Z = 14, 3920
    electrons), box padded by 10 bohr, graded degree-4 mesh of 36 x 36 x 36
    cells (1.28-bohr cells between the atom planes; 3,048,625 nodes), Slater
    1s/2s/2p enrichment (5 per atom, n_E = 1400), nuclear Coulomb plus a seeded
    32-term Gaussian perturbation; adaptive rule tau = 1e-7, depth <= 7 (46.7M
    quadrature points)."""
    atoms = diamond_cube_cut(3)
    Z = np.full(len(atoms), 14.0)
    return _cluster_system(atoms, Z, h_min, h_max, pad, r_c, seed, pot_seed, n_gaussians, tau, max_depth,
                           name=f"si{len(atoms)}")


def carbon_monoxide(h_min=1.0, h_max=3.0, pad=6.0, r_c=4.0, seed=12, tau=1e-7, max_depth=6):
    """C-O pair (Z = 6, 8; bond 2.132 bohr along x, 14 electrons) on a graded
    degree-4 mesh, Slater 1s/2s/2p enrichment (5 per atom, seeded exponents),
    bare nuclear potential: the small multi-atom system whose converged SCF the
    oracle provides for parity."""
    atoms = np.array([[0.0, 0.0, 0.0], [2.132, 0.0, 0.0]])
    return _cluster_system(atoms, np.array([6.0, 8.0]), h_min, h_max, pad, r_c, seed, seed + 1, 0, tau, max_depth,
                           name="co")


def _cluster_system(atoms, Z, h_min, h_max, pad, r_c, seed, pot_seed, n_gaussians, tau,
                    max_depth, name):
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = atoms.min(axis=0) - pad
    hi = atoms.max(axis=0) + pad
    breaks = [graded_breaks(lo[d], hi[d], atoms[:, d], h_min, h_max) for d in range(3)]
    funcs = []
    for ia, z in enumerate(Z):
        z1, z2 = slater_zetas(int(z))
        z1 *= 1.0 + 0.05 * rng.uniform(-1, 1)
        z2 *= 1.0 + 0.05 * rng.uniform(-1, 1)
        funcs += _slater_funcs(ia, z1, z2, r_c / 2.0, 1.0)
    prng = np.random.Generator(np.random.PCG64(pot_seed))
    amin, amax = atoms.min(axis=0), atoms.max(axis=0)
    pot = {"nuclear": True,
           "gauss_A": prng.uniform(-0.5, 0.5, size=n_gaussians),
           "gauss_s": prng.uniform(1.0, 3.0, size=n_gaussians),
           "gauss_c": amin + (amax - amin) * prng.uniform(0, 1, size=(n_gaussians, 3)),
           "omega": 0.0}
    return _system(breaks, 4, atoms, Z, funcs, pot, tau=tau, max_depth=max_depth, name=name)


def displaced_cluster(system, shift, h_min=1.0, h_max=3.5, pad=8.0, r_c=4.0, tau=1e-8, max_depth=7, seed=0):
    """The cluster of `system` with every atom moved by shift[I] (bohr, rounded to
    1e-3): same species, a new graded mesh around the new positions and the
    enrichment drawn with the same seeds as random_cluster(seed=seed)."""
    atoms = np.round(np.asarray(system["atoms"], dtype=np.float64) + np.asarray(shift, dtype=np.float64), 3)
    return _cluster_system(atoms, np.asarray(system["Z"], dtype=np.float64), h_min, h_max, pad, r_c, seed + 1000,
                           seed + 2000, 0, tau, max_depth, name=system["name"] + "_displaced")


def grid_dims(system):
    """Nodes per axis of the tensor-product node grid (boundary included)."""
    p = system["p"]
    return tuple(p * (len(b) - 1) + 1 for b in system["breaks"])


def n_nodes(system):
    nx, ny, nz = grid_dims(system)
    return nx * ny * nz


def boundary_mask(system):
    """True at nodes on the box faces (homogeneous Dirichlet rows)."""
    nx, ny, nz = grid_dims(system)
    ix = np.arange(nx)
    iy = np.arange(ny)
    iz = np.arange(nz)
    bx = (ix == 0) | (ix == nx - 1)
    by = (iy == 0) | (iy == ny - 1)
    bz = (iz == 0) | (iz == nz - 1)
    m = bz[:, None, None] | by[None, :, None] | bx[None, None, :]
    return m.reshape(-1)  # node index = ix + nx*(iy + ny*iz)


def initial_block(system, N, seed=1):
    """Initial subspace X0, rows = [all grid nodes; enrichment functions], N columns.

    Columns 0..min(N, n_E)-1 are unit vectors on the enrichment coefficients
    (the atomic orbitals themselves); the remaining columns are seeded normal
    random values on the interior nodes.  Boundary rows are zero."""
    nn = n_nodes(system)
    nE = len(system["funcs"])
    X = np.zeros((nn + nE, N))
    k = min(N, nE)
    for j in range(k):
        X[nn + j, j] = 1.0
    rng = np.random.Generator(np.random.PCG64(seed))
    if N > k:
        R = rng.standard_normal((nn, N - k))
        R[boundary_mask(system)] = 0.0
        X[:nn, k:] = R
    return X


def random_block(system, N, seed=5, scale=1.0):
    """Dense seeded random block (all interior and enrichment rows)."""
    nn = n_nodes(system)
    nE = len(system["funcs"])
    rng = np.random.Generator(np.random.PCG64(seed))
    X = scale * rng.standard_normal((nn + nE, N))
    X[:nn][boundary_mask(system)] = 0.0
    return X


def lanczos_start(system, seed=9):
    """Seeded start vector for the spectral upper-bound Lanczos run."""
    return random_block(system, 1, seed=seed)[:, 0].copy()

def sad_shells(Z):
    """Occupied shells (n, zeta, electrons) of a neutral atom for the superposition-
    of-atomic-densities start: 1s, 2s2p, 3s3p with Slater's-rules exponents
    (published screening constants 0.30 / 0.35 / 0.85 / 1.0)."""
    Z = int(Z)
    out = [(1, Z - 0.30 if Z > 1 else 1.0, float(min(Z, 2)))]
    if Z > 2:
        n2 = min(Z - 2, 8)
        out.append((2, (Z - (2 * 0.85 + (n2 - 1) * 0.35)) / 2.0, float(n2)))
    if Z > 10:
        n3 = min(Z - 10, 8)
        out.append((3, (Z - (2 * 1.0 + 8 * 0.85 + (n3 - 1) * 0.35)) / 3.0, float(n3)))
    return out


def random_cluster(n_atoms, species, seed, min_dist=3.0, density=0.012, h_min=1.0, h_max=3.5, pad=8.0,
                   r_c=4.0, tau=1e-8, max_depth=7):
    """Random non-overlapping cluster: Z drawn from `species`, positions uniform in a
    cube sized for about `density` atoms per bohr^3 with rejection to >= min_dist
    bohr spacing; graded degree-4 mesh, Slater 1s/2s/2p enrichment, no extra potential."""
    rng = np.random.Generator(np.random.PCG64(seed))
    side = (n_atoms / density) ** (1.0 / 3.0)
    pos = []
    while len(pos) < n_atoms:
        c = rng.uniform(0.0, side, size=3)
        if all(np.linalg.norm(c - q) >= min_dist for q in pos):
            pos.append(c)
    atoms = np.round(np.array(pos), 3)
    Z = rng.choice(np.asarray(species, dtype=np.float64), size=n_atoms)
    sysd = _cluster_system(atoms, Z, h_min, h_max, pad, r_c, seed + 1000, seed + 2000, 0, tau, max_depth,
                           name=f"cluster{n_atoms}_s{seed}")
    return sysd
