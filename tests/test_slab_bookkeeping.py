"""z-slab decomposition bookkeeping on the CPU: the partition of the planes, the ghost planes
and neighbours of every slab, and one halo exchange between two gloo ranks moving the right
planes to the right ghosts (a stand-in context whose planes carry their global z), with the
colour masses summed over the ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1804_08923_gb300 import slab
from paper_1804_08923_gb300._abi import BC_CONVECTIVE, BC_FREESLIP, BC_INLET, BC_PERIODIC


@pytest.mark.parametrize("nz,world", [(40, 2), (41, 3), (7, 3), (384, 8), (6, 3)])
def test_partition_covers_every_plane_once(nz, world):
    r = slab.partition(nz, world)
    assert r[0][0] == 0 and r[-1][1] == nz
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    sizes = [b - a for a, b in r]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 2


def test_partition_rejects_slabs_thinner_than_two_planes():
    with pytest.raises(ValueError):
        slab.partition(5, 3)


def test_geometry_of_an_inlet_outflow_lattice():
    bc = (BC_INLET, BC_CONVECTIVE)
    g = [slab.SlabGeometry(40, bc, r, 3) for r in range(3)]
    assert [(x.z0, x.z1) for x in g] == [(0, 14), (14, 27), (27, 40)]
    assert [x.bc[:2] for x in g] == [(BC_INLET, BC_FREESLIP), (BC_FREESLIP, BC_FREESLIP), (BC_FREESLIP, BC_CONVECTIVE)]
    assert [(x.lo, x.hi) for x in g] == [(False, True), (True, True), (True, False)]
    assert [x.nz_local for x in g] == [15, 15, 14]
    assert g[1].global_planes() == list(range(13, 28))
    assert g[0].transfers() == [(13, 1, 14, 1)] and g[2].transfers() == [(1, 1, 0, 0)]
    single = slab.SlabGeometry(40, bc, 0, 1)
    assert (single.nz_local, single.bc[:2], single.transfers()) == (40, bc, [])


def test_geometry_of_a_periodic_lattice_wraps():
    g = [slab.SlabGeometry(12, (BC_PERIODIC, BC_PERIODIC), r, 2) for r in range(2)]
    assert g[0].global_planes() == [11] + list(range(0, 6)) + [6]
    assert g[1].global_planes() == [5] + list(range(6, 12)) + [0]
    assert all(x.bc[:2] == (BC_FREESLIP, BC_FREESLIP) for x in g)
    assert g[0].below == g[0].above == 1


class PlaneContext:
    """Stand-in for a slab's context: every plane of every halo kind holds its global z (so
    a ghost shows where its contents came from) and a plane 'mass' of 1 + global z."""

    def __init__(self, geom, nbytes=(24, 8)):
        self.geom, self.nb = geom, nbytes
        zs = geom.global_planes()
        self.planes = {k: np.array([[z] * (n // 8) for z in zs], dtype=np.float64) for k, n in zip(slab.KINDS, nbytes)}
        self.calls = []

    def halo_bytes(self, kind):
        return self.nb[kind]

    def halo_pack(self, kind, z, buf):
        buf.view(np.float64)[:] = self.planes[kind][z]

    def halo_unpack(self, kind, z, buf):
        self.planes[kind][z] = buf.view(np.float64)

    def step_gather(self):
        self.calls.append("gather")

    def step_collide(self):
        self.calls.append("collide")

    def mass_planes(self, z0, z1):
        zs = np.array(self.geom.global_planes()[z0:z1], dtype=np.float64)
        return np.array([np.sum(1.0 + zs), 2.0 * len(zs)])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nz, bc, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = slab.SlabLattice((4, 3, nz), {}, bc, rank, world, dist, host_halos=True,
                         lattice_factory=lambda g, p, b: None)
    ctx = PlaneContext(s.geom)
    s.lat = ctx
    for k in slab.KINDS:  # poison the ghost planes: the exchange must overwrite them
        if s.geom.lo:
            ctx.planes[k][0] = -1.0
        if s.geom.hi:
            ctx.planes[k][-1] = -1.0
    s.step(2)
    ghosts = {k: (ctx.planes[k][0][0], ctx.planes[k][-1][0]) for k in slab.KINDS}
    q.put((rank, s.geom.global_planes(), ghosts, ctx.calls, s.mass().tolist()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("bc", [(BC_INLET, BC_CONVECTIVE), (BC_PERIODIC, BC_PERIODIC)])
def test_two_gloo_ranks_exchange_the_boundary_planes(bc):
    nz, world = 10, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, nz, bc, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, zs, ghosts, calls, mass in res:
        assert calls == ["gather", "collide"] * 2
        for k in slab.KINDS:
            assert ghosts[k] == (float(zs[0]), float(zs[-1]))  # every ghost holds its global plane
        # the whole lattice's masses: sum over z of 1 + z, and 2 per plane
        assert mass == [float(sum(1 + z for z in range(nz))), 2.0 * nz]
