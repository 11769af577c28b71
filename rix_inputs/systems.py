"""Synthetic geometries, species tables and auxiliary-basis widths.

Five workloads stand in for the paper's benchmark structures (the paper's
water, ice and hybrid-perovskite systems, Sec. "Benchmark calculations for
selected systems"; their NOMAD/ELSI geometries are not available):

  0  (H2O)_8 cluster, molecules on a 2.8 A cubic lattice, no cutoff
  1  (H2O)_64 cluster, same generators, 8 A cutoff, screening 1e-10
  2  ice-like periodic cell, 256 H2O (4x2x4 orthorhombic ice-XI cells)
  3  perovskite-like periodic cell, 1536 atoms, 6.3 A Pb-Pb spacing
  4  ice-like periodic cell, 1024 H2O (8x4x4 orthorhombic ice-XI cells)

The oxygen sublattice of the ice cells is the ice-XI primitive cell printed
in the paper's supplementary information ("Supercell of Ice XI"), converted
to its orthorhombic setting and rescaled to 0.92 g/cm^3.  Hydrogens get a
random molecular orientation (no ice rules).

All coordinates are returned in bohr.
"""
from dataclasses import dataclass, field
import numpy as np

from . import rng

ANGSTROM_PER_BOHR = 0.529177210903
OMEGA = 0.11  # range-separation parameter of HSE06, bohr^-1
CUTOFF_ANGSTROM = 8.0
D_SUPPORT_ANGSTROM = 4.0
SCREEN_TAU = 1e-10

# (basis functions, auxiliary functions) per species
SPECIES_SIZES = {
    "O": (14, 56), "H": (5, 16), "Pb": (39, 140), "I": (32, 120),
    "C": (14, 56), "N": (14, 56),
}
VALENCE = {"Pb": 4, "I": 7, "C": 4, "N": 5, "H": 1, "O": 6}


def ang2bohr(x):
    return np.asarray(x, dtype=np.float64) / ANGSTROM_PER_BOHR


@dataclass
class System:
    name: str
    seed: int
    xyz: np.ndarray                 # [n,3] bohr
    species: np.ndarray             # [n] int32 index into species_names
    species_names: list
    nbas: np.ndarray                # [n_species] int32
    naux: np.ndarray                # [n_species] int32
    sigma: list                     # per species: [naux] aux widths (bohr), ascending
    cell: np.ndarray = None         # [3,3] rows are lattice vectors (bohr); None = cluster
    cutoff: float = 0.0             # bohr; <= 0 means no cutoff
    tau: float = 0.0                # block screening threshold; <= 0 means none
    orbital_centres: np.ndarray = None  # [n_occ] atom index of each occupied orbital centre
    meta: dict = field(default_factory=dict)
    omega: float = OMEGA            # range separation of V (bohr^-1); <= 0: full-range Coulomb (PBE0)

    @property
    def n_atoms(self):
        return int(self.xyz.shape[0])

    def nb_atom(self):
        return self.nbas[self.species]

    def na_atom(self):
        return self.naux[self.species]

    @property
    def nbasis(self):
        return int(self.nb_atom().sum())

    @property
    def nauxtot(self):
        return int(self.na_atom().sum())


def _quaternion_rotations(u):
    """Uniform random rotations from uniforms u[...,3] (Shoemake 1992)."""
    u1, u2, u3 = u[:, 0], u[:, 1], u[:, 2]
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], axis=1)
    x, y, z, w = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((len(u), 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _water_template():
    """O at origin, two H at 0.96 A with a 104.5 degree H-O-H angle (A)."""
    th = np.deg2rad(104.5) / 2
    r = 0.96
    return np.array([[0.0, 0.0, 0.0],
                     [r * np.sin(th), 0.0, r * np.cos(th)],
                     [-r * np.sin(th), 0.0, r * np.cos(th)]])


def _aux_widths(seed, names):
    """Per-species aux widths, log-uniform in [0.3, 3] bohr, sorted ascending."""
    out = []
    for s, nm in enumerate(names):
        na = SPECIES_SIZES[nm][1]
        u = rng.uniform(seed, rng.STREAM_AUX, np.arange(na) + 4096 * s)
        out.append(np.sort(0.3 * np.exp(u * np.log(10.0))))
    return out


def _species_arrays(names):
    nb = np.array([SPECIES_SIZES[n][0] for n in names], dtype=np.int32)
    na = np.array([SPECIES_SIZES[n][1] for n in names], dtype=np.int32)
    return nb, na


def _waters(o_pos_ang, seed):
    """Place a randomly oriented water on every O site; atoms ordered O,H,H."""
    nmol = len(o_pos_ang)
    u = rng.uniform(seed, rng.STREAM_GEOM, np.arange(3 * nmol)).reshape(nmol, 3)
    R = _quaternion_rotations(u)
    tmpl = _water_template()
    xyz = o_pos_ang[:, None, :] + np.einsum("mij,aj->mai", R, tmpl)
    species = np.tile(np.array([0, 1, 1], dtype=np.int32), nmol)
    return xyz.reshape(-1, 3), species


def water_cluster(n_side, seed, cutoff=True):
    g = np.arange(n_side) * 2.8
    o = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    xyz, species = _waters(o, seed)
    names = ["O", "H"]
    nb, na = _species_arrays(names)
    return System(
        name=f"(H2O)_{len(o)} cluster", seed=seed, xyz=ang2bohr(xyz), species=species,
        species_names=names, nbas=nb, naux=na, sigma=_aux_widths(seed, names),
        cell=None,
        cutoff=ang2bohr(CUTOFF_ANGSTROM) if cutoff else 0.0,
        tau=SCREEN_TAU if cutoff else 0.0,
        orbital_centres=np.repeat(np.arange(0, len(species), 3), 5).astype(np.int32),
        meta={"kind": "water-cluster", "n_molecules": len(o)},
    )


# Ice-XI primitive cell from the supplementary information (A and fractional O).
_ICE_A1 = np.array([2.1246016568898547, -3.6755729842109162, 0.0])
_ICE_A2 = np.array([2.1246016568898547, 3.6755729842109162, 0.0])
_ICE_A3 = np.array([0.0, 0.0, 6.9422303803022247])
_ICE_O_FRAC = np.array([
    [0.1796291960199634, 0.8203708039800366, 0.4413296411621622],
    [0.8203708039800366, 0.1796291960199634, 0.9413296411621622],
    [0.8458673171536840, 0.1541326828463160, 0.5672469013890502],
    [0.1541326828463159, 0.8458673171536841, 0.0672469013890502],
])
WATER_MASS_AMU = 18.01528
AVOGADRO = 6.02214076e23


def ice_orthorhombic_cell(density=0.92):
    """Orthorhombic ice-XI cell (8 O) rescaled to the given density; returns (abc_A, O_xyz_A)."""
    A = _ICE_A1 + _ICE_A2
    B = _ICE_A2 - _ICE_A1
    C = _ICE_A3
    abc = np.array([A[0], B[1], C[2]])
    prim = _ICE_O_FRAC @ np.stack([_ICE_A1, _ICE_A2, _ICE_A3])
    o = np.concatenate([prim, prim + _ICE_A1])
    o = np.mod(o, abc)
    vol = abc.prod() * 1e-24  # cm^3
    rho = 8 * WATER_MASS_AMU / AVOGADRO / vol
    s = (rho / density) ** (1.0 / 3.0)
    return abc * s, o * s


def ice(nx, ny, nz, seed):
    abc, o_cell = ice_orthorhombic_cell()
    shifts = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"),
                      axis=-1).reshape(-1, 3) * abc
    o = (shifts[:, None, :] + o_cell[None, :, :]).reshape(-1, 3)
    xyz, species = _waters(o, seed)
    names = ["O", "H"]
    nb, na = _species_arrays(names)
    cell = np.diag(abc * np.array([nx, ny, nz]))
    return System(
        name=f"ice-like {len(o)} H2O ({nx}x{ny}x{nz} cells)", seed=seed, xyz=ang2bohr(xyz),
        species=species, species_names=names, nbas=nb, naux=na,
        sigma=_aux_widths(seed, names), cell=ang2bohr(cell),
        cutoff=ang2bohr(CUTOFF_ANGSTROM), tau=SCREEN_TAU,
        orbital_centres=np.repeat(np.arange(0, len(species), 3), 5).astype(np.int32),
        meta={"kind": "ice", "n_molecules": len(o), "cell_A": (abc * [nx, ny, nz]).tolist()},
    )


def _largest_remainder(total, weights):
    w = np.asarray(weights, dtype=np.float64)
    exact = total * w / w.sum()
    base = np.floor(exact).astype(int)
    rem = total - base.sum()
    order = np.argsort(-(exact - base), kind="stable")
    base[order[:rem]] += 1
    return base


def perovskite(nx, ny, nz, seed, a=6.3):
    """Pb on a cubic lattice, I at a/2 along each axis, 8 organics per A-site cavity."""
    names = ["Pb", "I", "C", "N", "H"]
    ncell = nx * ny * nz
    n_org = 8 * ncell
    counts = _largest_remainder(n_org, [2, 1, 8])  # C, N, H
    org_species = np.concatenate([np.full(counts[0], 2), np.full(counts[1], 3),
                                  np.full(counts[2], 4)]).astype(np.int32)
    # draw order on the geometry stream: species shuffle, organic positions, jitter
    c0 = 0
    perm = np.argsort(rng.uniform(seed, rng.STREAM_GEOM, c0 + np.arange(n_org)), kind="stable")
    c0 += n_org
    org_species = org_species[perm]
    u = rng.uniform(seed, rng.STREAM_GEOM, c0 + np.arange(3 * n_org)).reshape(n_org, 3)
    c0 += 3 * n_org
    # uniform point in a ball of radius 1.5 A: radius r = 1.5 u^(1/3), direction uniform
    r = 1.5 * np.cbrt(u[:, 0])
    cz = 2.0 * u[:, 1] - 1.0
    ph = 2.0 * np.pi * u[:, 2]
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    org_off = np.stack([r * sz * np.cos(ph), r * sz * np.sin(ph), r * cz], axis=1)
    xyz, species = [], []
    k = 0
    for ix in range(nx):
        for iy in range(ny):
            for iz in range(nz):
                p = np.array([ix, iy, iz], dtype=np.float64) * a
                xyz.append(p); species.append(0)
                for d in range(3):
                    e = np.zeros(3); e[d] = a / 2
                    xyz.append(p + e); species.append(1)
                centre = p + a / 2
                for _ in range(8):
                    xyz.append(centre + org_off[k]); species.append(int(org_species[k])); k += 1
    xyz = np.array(xyz)
    species = np.array(species, dtype=np.int32)
    jit = 0.1 * rng.normal(seed, rng.STREAM_GEOM, c0 + np.arange(xyz.size)).reshape(xyz.shape)
    xyz = xyz + jit
    nb, na = _species_arrays(names)
    # occupied orbitals: floor(v/2) on every atom, odd-valence atoms paired in index order
    cent = []
    odd = []
    for i, s in enumerate(species):
        v = VALENCE[names[s]]
        cent.extend([i] * (v // 2))
        if v % 2:
            odd.append(i)
    cent.extend(odd[0::2][: len(odd) // 2])
    cell = np.diag(np.array([nx, ny, nz], dtype=np.float64) * a)
    comp = {nm: int((species == s).sum()) for s, nm in enumerate(names)}
    return System(
        name=f"perovskite-like {len(species)} atoms ({nx}x{ny}x{nz} cells)", seed=seed,
        xyz=ang2bohr(xyz), species=species, species_names=names, nbas=nb, naux=na,
        sigma=_aux_widths(seed, names), cell=ang2bohr(cell),
        cutoff=ang2bohr(CUTOFF_ANGSTROM), tau=SCREEN_TAU,
        orbital_centres=np.array(cent, dtype=np.int32),
        meta={"kind": "perovskite", "composition": comp, "n_occ": len(cent)},
    )


CONFIG_NAMES = {
    0: "(H2O)8 cluster, 24 atoms, no cutoff",
    1: "(H2O)64 cluster, 192 atoms, 8 A cutoff",
    2: "ice-like periodic, 768 atoms, 8 A images",
    3: "perovskite-like periodic, 1536 atoms, 8 A images",
    4: "ice-like periodic, 3072 atoms, 8 A images",
}


def full_range(system):
    """The same workload with the full-range Coulomb metric of PBE0 (omega -> 0) instead of HSE06's."""
    import dataclasses
    return dataclasses.replace(system, name=system.name + " (PBE0 kernel)", omega=0.0)


def config(i):
    """The five synthetic workloads; seed = config index."""
    if i == 0:
        return water_cluster(2, seed=0, cutoff=False)
    if i == 1:
        return water_cluster(4, seed=1)
    if i == 2:
        return ice(4, 2, 4, seed=2)
    if i == 3:
        return perovskite(8, 4, 4, seed=3)
    if i == 4:
        return ice(8, 4, 4, seed=4)
    raise ValueError(i)
