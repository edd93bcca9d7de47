"""z-slab decomposition of one lattice over several contexts.

The step is a nearest-neighbour stencil in z, so a lattice splits into slabs of consecutive
planes.  Each slab is an ordinary context (``Lattice``) holding its real planes plus one ghost
plane on every side that borders another slab; twice per step the ghost planes receive the
neighbour's boundary plane (populations before the gather pass, phase entries before the
collision), see the z-slab section of ``include/lbcm.h``.  The real planes then evolve bit for
bit as the same planes of the whole lattice.

``SlabLattice`` is one slab of a job whose ranks exchange halos through ``torch.distributed``
(point-to-point send/receive of one plane per neighbour and kind; NCCL with device buffers,
gloo with host buffers); colour masses are summed over the ranks in FP64.  ``SlabGroup`` steps
several slabs held by one process (one or several GPUs) with device-to-device halo copies.
This module only moves planes and arguments; the arithmetic is the library's.
"""
from __future__ import annotations

import numpy as np

from ._abi import BC_FREESLIP, BC_PERIODIC, HALO_PHASE, HALO_POPULATIONS

KINDS = (HALO_POPULATIONS, HALO_PHASE)


def partition(nz: int, world: int):
    """Plane ranges [z0, z1) of the slabs: consecutive, covering [0, nz), sizes differing by at
    most one (the first nz % world slabs one plane longer).  Every slab needs two real planes
    (the convective outflow reads the plane below the last one)."""
    if world < 1 or nz < 2 * world:
        raise ValueError(f"{nz} planes cannot be split into {world} slabs of at least two planes")
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


class SlabGeometry:
    """Where slab `rank` of `world` sits: its real planes [z0, z1) of the whole lattice, its
    ghost planes, its neighbours and the boundaries its own context takes."""

    def __init__(self, nz: int, bc, rank: int, world: int):
        bc = tuple(bc) + (BC_PERIODIC, BC_PERIODIC)[len(bc) - 2:] if len(bc) < 4 else tuple(bc)
        self.nz, self.rank, self.world = nz, rank, world
        self.z0, self.z1 = partition(nz, world)[rank]
        periodic = bc[0] == BC_PERIODIC
        split = world > 1
        self.lo = split and (rank > 0 or periodic)  # ghost plane below the first real plane
        self.hi = split and (rank < world - 1 or periodic)
        self.below = (rank - 1) % world if self.lo else None  # neighbour ranks
        self.above = (rank + 1) % world if self.hi else None
        self.nz_local = (self.z1 - self.z0) + int(self.lo) + int(self.hi)
        self.first = int(self.lo)  # local index of the first real plane
        self.last = self.nz_local - 1 - int(self.hi)  # ... of the last real plane
        zlo = BC_FREESLIP if self.lo else bc[0]
        zhi = BC_FREESLIP if self.hi else bc[1]
        self.bc = (zlo, zhi, bc[2], bc[3])

    def global_planes(self):
        """Global z of every local plane (ghosts wrap where the lattice is periodic)."""
        return [(self.z0 - int(self.lo) + k) % self.nz for k in range(self.nz_local)]

    def transfers(self):
        """(local plane sent, neighbour, local ghost plane received, tag side) of one exchange:
        the first real plane goes down and the plane below comes up into ghost 0, the last real
        plane goes up and the plane above comes down into the top ghost."""
        out = []
        if self.lo:
            out.append((self.first, self.below, 0, 0))
        if self.hi:
            out.append((self.last, self.above, self.nz_local - 1, 1))
        return out


def _local_fields(geom: SlabGeometry, rho_r, rho_b, u):
    zs = geom.global_planes()
    return (np.ascontiguousarray(np.asarray(rho_r)[zs]), np.ascontiguousarray(np.asarray(rho_b)[zs]),
            np.ascontiguousarray(np.asarray(u)[:, zs]))


class SlabLattice:
    """Slab `rank` of a lattice split over `world` ranks of a torch.distributed group.

    lattice_factory(grid, params, bc) makes the slab's context (default: the CUDA ``Lattice``
    on `device`); host_halos exchanges through host buffers (gloo), else through device
    buffers (NCCL)."""

    def __init__(self, grid, params: dict, bc, rank: int, world: int, dist, device=None, host_halos=False,
                 lattice_factory=None):
        nx, ny, nz = (int(v) for v in grid)
        self.geom = SlabGeometry(nz, bc, rank, world)
        self.dist, self.host = dist, host_halos
        if lattice_factory is None:
            from . import Lattice
            lattice_factory = lambda g, p, b: Lattice(g, p, bc=b, device=device)  # noqa: E731
        self.lat = lattice_factory((nx, ny, self.geom.nz_local), params, self.geom.bc)
        self.device = device
        self._bufs = {}

    # ------------------------------------------------------------------ halos
    def _buf(self, kind, side, direction):
        key = (kind, side, direction)
        if key not in self._bufs:
            import torch
            n = self.lat.halo_bytes(kind)
            dev = "cpu" if self.host else self.device
            self._bufs[key] = torch.empty(n, dtype=torch.uint8, device=dev)
        return self._bufs[key]

    def exchange(self, kind):
        """One halo exchange of `kind` with both neighbours (non-blocking sends and receives,
        then the unpacks)."""
        import torch
        reqs, recv = [], []
        for plane, peer, ghost, side in self.geom.transfers():
            out = self._buf(kind, side, 0)
            self.lat.halo_pack(kind, plane, out if not self.host else out.numpy())
            if not self.host:
                torch.cuda.current_stream().wait_stream(self.lat.stream)
            inc = self._buf(kind, side, 1)
            # tag: kind and the side the plane travels to, so the two messages between the same
            # pair of ranks (world == 2 with periodic z) cannot be confused
            reqs.append(self.dist.isend(out, dst=peer, tag=2 * kind + side))
            reqs.append(self.dist.irecv(inc, src=peer, tag=2 * kind + (1 - side)))
            recv.append((ghost, inc))
        for r in reqs:
            r.wait()
        for ghost, inc in recv:
            if not self.host:
                self.lat.stream.wait_stream(torch.cuda.current_stream())
            self.lat.halo_unpack(kind, ghost, inc if not self.host else inc.numpy())

    # ------------------------------------------------------------------ stepping
    def step(self, n=1):
        for _ in range(n):
            self.exchange(HALO_POPULATIONS)
            self.lat.step_gather()
            self.exchange(HALO_PHASE)
            self.lat.step_collide()

    def init_jet(self):
        self.lat.init_jet()

    def init_fields(self, rho_r, rho_b, u):
        """Fields of the whole lattice, (nz, ny, nx) and (3, nz, ny, nx): each slab takes its own
        planes and its ghosts'."""
        self.lat.init_fields(*_local_fields(self.geom, rho_r, rho_b, u))

    # ------------------------------------------------------------------ outputs
    def populations(self):
        """Populations of the real planes, (2, 27, z1 - z0, ny, nx) float32 numpy."""
        return self.lat.populations(device=False)[:, :, self.geom.first:self.geom.last + 1]

    def mass(self):
        """Colour masses of the whole lattice: FP64 sums of the real planes, summed over the
        ranks in FP64."""
        import torch
        m = self.lat.mass_planes(self.geom.first, self.geom.last + 1)
        t = torch.tensor(m, dtype=torch.float64, device="cpu" if self.host else self.device)
        self.dist.all_reduce(t)
        return t.cpu().numpy()


class SlabGroup:
    """Several slabs of one lattice held by this process (on one GPU or several), stepped in
    lockstep; halos move by device-to-device copies."""

    def __init__(self, grid, params: dict, bc, world: int, devices=None):
        from . import Lattice
        nx, ny, nz = (int(v) for v in grid)
        devices = devices or ["cuda"] * world
        self.geoms = [SlabGeometry(nz, bc, r, world) for r in range(world)]
        self.lats = [Lattice((nx, ny, g.nz_local), params, bc=g.bc, device=d) for g, d in zip(self.geoms, devices)]

    def exchange(self, kind):
        import torch
        planes = []
        for g, lat in zip(self.geoms, self.lats):
            for plane, peer, ghost, side in g.transfers():
                buf = torch.empty(lat.halo_bytes(kind), dtype=torch.uint8, device=lat.device)
                lat.halo_pack(kind, plane, buf)
                planes.append((peer, side, buf, lat))
        for src_lat in self.lats:
            src_lat.stream.synchronize()
        for peer, side, buf, _ in planes:
            g, lat = self.geoms[peer], self.lats[peer]
            ghost = g.nz_local - 1 if side == 0 else 0  # sent down: the receiver's top ghost
            lat.halo_unpack(kind, ghost, buf.to(lat.device))
        for lat in self.lats:
            lat.stream.synchronize()

    def step(self, n=1):
        for _ in range(n):
            self.exchange(HALO_POPULATIONS)
            for lat in self.lats:
                lat.step_gather()
            self.exchange(HALO_PHASE)
            for lat in self.lats:
                lat.step_collide()

    def init_jet(self):
        for lat in self.lats:
            lat.init_jet()

    def init_fields(self, rho_r, rho_b, u):
        for g, lat in zip(self.geoms, self.lats):
            lat.init_fields(*_local_fields(g, rho_r, rho_b, u))

    def populations(self):
        """Populations of the whole lattice joined from the slabs' real planes."""
        return np.concatenate([lat.populations(device=False)[:, :, g.first:g.last + 1]
                               for g, lat in zip(self.geoms, self.lats)], axis=2)

    def mass(self):
        return np.sum([lat.mass_planes(g.first, g.last + 1) for g, lat in zip(self.geoms, self.lats)], axis=0)

    def close(self):
        for lat in self.lats:
            lat.close()
