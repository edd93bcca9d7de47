"""z-slab decomposition on the GPU: a lattice split into slabs (each its own context with
ghost planes, halos exchanged twice per step) evolves bit for bit as the whole lattice.

In one process (SlabGroup, every slab on cuda:0, device-to-device halo copies) and as two
gloo ranks that share cuda:0 and exchange through host buffers (SlabLattice); the ranks'
kernels never wait on one another: every exchange happens on the host between launches."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_08923_gb300.build as b
    b.build()
    import paper_1804_08923_gb300 as lbm
    return lbm


def jet(storage=0):
    cfg = workloads.scaled_jet("jet96", 36, 34, 40, D=10)
    return (36, 34, 40), tuple(cfg["bc"]), dict(cfg["params"], storage=storage)


@pytest.mark.parametrize("world,storage", [(2, 0), (3, 0), (2, 1), (3, 2)])
def test_split_jet_equals_the_whole_lattice(lb, world, storage):
    """Inlet disc with noise (first slab), convective outflow (last slab), 50 steps."""
    from paper_1804_08923_gb300 import slab
    grid, bc, params = jet(storage)
    whole = lb.Lattice(grid, params, bc=bc)
    whole.init_jet()
    whole.step(50)
    group = slab.SlabGroup(grid, params, bc, world)
    group.init_jet()
    group.step(50)
    assert np.array_equal(group.populations(), whole.populations(device=False))
    assert np.allclose(group.mass(), whole.mass(), rtol=1e-12, atol=0)
    assert whole.fields(device=False)["rho_r"].sum() > 0.5  # red has entered
    group.close()


def test_split_periodic_two_phase_with_gravity(lb):
    """Periodic z (every slab has two ghosts; the end slabs are neighbours), a random two-phase
    state with gravity and density contrast, three slabs, 40 steps."""
    from paper_1804_08923_gb300 import slab
    nx, ny, nz = 20, 9, 18
    params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.08, sigma=0.003, g=(1e-6, 0.0, 1e-5))
    fields = workloads.random_two_phase_fields((nz, ny, nx), 3, 1.0, 0.5, u_amp=0.03)
    whole = lb.Lattice((nx, ny, nz), params)
    whole.init_fields(*fields)
    whole.step(40)
    group = slab.SlabGroup((nx, ny, nz), params, (0, 0), 3)
    group.init_fields(*fields)
    group.step(40)
    assert np.array_equal(group.populations(), whole.populations(device=False))
    group.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    import paper_1804_08923_gb300 as lbm
    from paper_1804_08923_gb300 import slab
    grid, bc, params = jet()
    s = slab.SlabLattice(grid, params, bc, rank, world, dist, device="cuda:0", host_halos=True)
    s.init_jet()
    s.step(50)
    mine = s.populations()
    mass = s.mass()
    whole = lbm.Lattice(grid, params, bc=bc)
    whole.init_jet()
    whole.step(50)
    ref = whole.populations(device=False)[:, :, s.geom.z0:s.geom.z1]
    q.put((rank, bool(np.array_equal(mine, ref)), bool(np.allclose(mass, whole.mass(), rtol=1e-12, atol=0))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu_equal_the_whole_lattice(lb):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res == [(0, True, True), (1, True, True)], res


def test_split_step_order_is_enforced(lb):
    grid, bc, params = jet()
    lat = lb.Lattice(grid, params, bc=bc)
    lat.init_jet()
    with pytest.raises(lb.LBError):
        lat.step_collide()
    lat.step_gather()
    with pytest.raises(lb.LBError):
        lat.step(1)
    with pytest.raises(lb.LBError):
        lat.step_gather()
    import numpy as np_
    buf = np_.zeros(lat.halo_bytes(0), np_.uint8)
    with pytest.raises(lb.LBError):
        lat.halo_pack(0, 3, buf)  # population halo inside a split step
    lat.step_collide()
    with pytest.raises(lb.LBError):
        lat.halo_pack(1, 3, np_.zeros(lat.halo_bytes(1), np_.uint8))  # phase halo outside one
    with pytest.raises(lb.LBError):
        lat.halo_pack(0, 40, buf)  # plane outside the lattice
    assert lat.step_count == 1
