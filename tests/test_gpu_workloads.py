"""The mixed-precision path on the full-size periodic workloads, against the oracle.

Workloads (the same seeded generators as everywhere else):
* ice-like cell, 768 atoms (256 H2O), nbasis 6,144;
* perovskite-like cell, 1,536 atoms (Pb/I/C/N/H), nbasis 24,911, C = 70.7 GB;
* ice-like supercell, 3,072 atoms (1,024 H2O), nbasis 24,576, C = 24.6 GB.

The oracle cannot build all of K for these cells in test time, so each check
uses what it can compute exactly:
* K blocks sampled from a few row atoms of every species (the oracle's
  block-sampled build: T and Z restricted to the nodes those blocks need),
  relative Frobenius error of the mixed path <= 1e-8;
* whole K rows of a few row atoms (the oracle's row mode) and their energies
  -1/4 sum <D(E,A,-n), K(A,E,n)>: every sampled row's energy within
  1e-6 Ha / sqrt(n_atoms) of the oracle's.  E_x is the sum of n_atoms row
  energies whose rounding errors (from the slice truncation, of either sign)
  add up like a random walk: rows at that level give |dE_x| ~ 1e-6 Ha.  (The
  measured row errors sit 30-100x below it; the full E_x of the 3,072-atom
  cell is compared with the FP64 path in the benchmark line.)
* on the 768-atom cell, where the FP64 build takes seconds, E_x of the mixed
  path within 1e-6 Ha of the FP64 path's, whose rows match the oracle to 1e-12
  (tests/test_gpu_fp64.py).
C and V are loaded from host memory (rix_set_CV accepts host pointers), so the
device holds one copy of C.
"""
import time

import numpy as np
import pytest

import rix_inputs as ri
from oracle.oracle import Oracle
from workloads import gather_blocks, k_offsets, rel, row_energies, rows_of, sample_keys

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300.rix import Exchange  # noqa: E402

K_TOL = 1e-8
E_TOL_HA = 1e-6
GB = 1 << 30

# row atoms whose whole K rows the oracle builds: a water (O, H, H) / an H and a C of the perovskite
ROWS = {2: [300, 301, 302], 3: None, 4: [1536, 1537, 1538]}


def _perovskite_rows(s):
    names = list(s.species_names)
    h = int(np.nonzero(s.species == names.index("H"))[0][0])
    c = int(np.nonzero(s.species == names.index("C"))[0][0])
    return sorted([c, h])


def _mixed(s, pk):
    cap = int(torch.cuda.mem_get_info()[0] - 12 * GB)   # room for D, K and the caller's tensors
    ex = Exchange.from_system(s, precision="mixed", max_workspace_bytes=cap)
    ex.set_CV(pk.C, pk.V)
    D = torch.from_numpy(pk.D).cuda()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    K = ex.build_K(D)
    E = ex.energy(D, K)
    ev[1].record()
    torch.cuda.synchronize()
    keys = ex.k_keys()
    st = ex.stats()
    print(f"[{s.name}] mixed build + energy {ev[0].elapsed_time(ev[1]) / 1e3:.2f} s, "
          f"{st['n_row_blocks']} row block(s), workspace {st['workspace_bytes'] / GB:.1f} GiB", flush=True)
    Kh = K.cpu().numpy()
    ex.close()
    del K, D
    torch.cuda.empty_cache()
    return keys, Kh, E.item()


@pytest.mark.parametrize("cfg", [2, 4, 3])
def test_mixed_workload_against_oracle(cfg):
    s = ri.config(cfg)
    t0 = time.time()
    pk = ri.generate(s)
    print(f"[{s.name}] inputs in {time.time() - t0:.1f} s, C {pk.C.nbytes / 1e9:.1f} GB", flush=True)
    keys, K, E = _mixed(s, pk)
    off = k_offsets(s, keys)
    orc = Oracle(s)
    orc.set_data(pk.C, pk.V, pk.D)
    assert np.array_equal(orc.kpattern(), keys), "K pattern differs from the oracle's"
    # sampled blocks of every species
    t0 = time.time()
    want = sample_keys(s, keys, np.random.default_rng(cfg))
    kk = orc.kpattern_blocks(want)
    Kref = orc.build_K()
    assert np.array_equal(kk, want)
    eb = rel(gather_blocks(keys, off, K, kk), Kref)
    print(f"[{s.name}] {len(kk)} sampled blocks: mixed vs oracle {eb:.2e} ({time.time() - t0:.1f} s)", flush=True)
    assert eb < K_TOL
    # whole rows and their energies
    rows = ROWS[cfg] if ROWS[cfg] is not None else _perovskite_rows(s)
    t0 = time.time()
    kr = orc.kpattern(rows)
    Kr = orc.build_K()
    e_ref = orc.energy(Kr, per_row=True)[1]
    sub_keys, sub = rows_of(s, keys, K, rows)
    assert np.array_equal(sub_keys, kr)
    er = rel(sub, Kr)
    e_got, _ = row_energies(s, pk, keys, K, rows)
    de = np.abs(e_got - e_ref)
    print(f"[{s.name}] rows {rows}: K {er:.2e}, row energies |dE| max {de.max():.2e} Ha "
          f"({time.time() - t0:.1f} s); E_x {E:.10f} Ha", flush=True)
    assert er < K_TOL
    assert (de < E_TOL_HA / np.sqrt(s.n_atoms)).all()
    if cfg == 2:
        ex = Exchange.from_system(s)
        ex.set_CV(pk.C, pk.V)
        D = torch.from_numpy(pk.D).cuda()
        E64 = ex.energy(D, ex.build_K(D)).item()
        ex.close()
        print(f"[{s.name}] E_x mixed - FP64 {E - E64:.3e} Ha", flush=True)
        assert abs(E - E64) < E_TOL_HA
