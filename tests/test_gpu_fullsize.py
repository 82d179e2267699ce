"""Parity at full size, in the launch configuration the benchmark times.

* 128^3 D3Q19 droplet (the benchmark workload, default kernel and tiles): after
  a few fused steps, one more step on the GPU is compared with the FP64 oracle
  evaluated site by site (oracle.step_sites) on a seeded sample of sites that
  includes every face, edge and corner region of the periodic box.
* 512^3 (the largest workload): properties that hold at any size -- per
  component mass conservation and total momentum conservation (section 2)."""
import numpy as np
import pytest

import oracle
import sc_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2112_02574_gb300 import binding

    return binding


def sample_sites(shape, n, seed=7):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    xs = np.concatenate([rng.integers(0, nx, n), [0, nx - 1, 0, nx - 1, 31, 32, 63, 64]])
    ys = np.concatenate([rng.integers(0, ny, n), [0, ny - 1, ny - 1, 0, 3, 4, 127, 0]])
    zs = np.concatenate([rng.integers(0, nz, n), [0, nz - 1, nz - 1, 0, 15, 16, 17, 127]])
    return xs + nx * (ys + ny * zs)


def test_bench_workload_one_step_sampled(B):
    shape = (128, 128, 128)
    nA0, nB0 = S.droplet(shape[::-1], (64, 64, 64), 24.0, n_in=0.95, n_out=0.05, amplitude=1e-3)
    p = B.make_params(shape, lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=B.SC_STORE_F32, G=3.6)
    sim = B.Simulation(p, nA0, nB0)
    sim.step(20)
    f = sim.populations().cpu().numpy()
    sim.step(1)
    sim.sync()
    f1 = sim.populations().cpu().numpy()
    op = oracle.Params(shape=shape, lattice=oracle.D3Q19, psi_self=oracle.PSI_EXP, G=3.6)
    sites = sample_sites(shape, 1500)
    want = oracle.step_sites(op, f, sites)
    got = f1[:, :, sites]
    # one FP32 step from an exactly representable state: FP32 round-off only
    assert np.abs(got - want).max() < 1e-6 * np.abs(want).max()
    nA, nB, _ = sim.moments(with_u=False)
    assert abs(nA.sum().item() - nA0.sum()) < 1e-6 * nA0.sum()


def test_largest_lattice_conservation(B):
    import torch

    shape = (512, 512, 512)
    free, _ = torch.cuda.mem_get_info()
    p = B.make_params(shape, lattice=B.SC_D3Q19, psi_self=B.SC_PSI_EXP, storage=B.SC_STORE_F32, G=3.6,
                      G_self=(-0.6, 0.0))
    if B.sc_workspace_bytes(p) + (8 << 30) > free:
        pytest.skip("not enough free device memory for the 512^3 lattice")
    nA0, nB0 = S.droplet(shape[::-1], (256, 256, 256), 96.0, n_in=0.95, n_out=0.05, amplitude=1e-3)
    sim = B.Simulation(p, nA0, nB0)
    del nA0, nB0
    t0 = sim.totals().cpu().numpy()
    sim.step(4)
    sim.sync()
    t1 = sim.totals().cpu().numpy()
    assert np.abs(t1[:2] - t0[:2]).max() < 1e-6 * t0[:2].max()
    assert np.abs(t1[2:]).max() < 1e-6 * t0[:2].sum()
