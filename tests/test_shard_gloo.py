"""The partitioned substep (sources traced by their owner process, cells
integrated by the owner of their z-slab; Sect. 5) on two CPU processes over
gloo, with the FP64 oracle doing each process's share: after A3 and A2
substeps with Eq. 4 steps, both processes hold exactly the state of the
single-process oracle run.  This checks what the exchanges must carry and
in which order (columns of every source before the dt pass and the full
step, slabs of x_half before the second trace, slabs of x at the end, the
minimum of the dt values), without a GPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    from paper_1201_5651_gb300 import inputs
    w = inputs.small_random(n=11, ny=9, nz=10, seed=73, nsrc=4, spectrum="bb")
    return w


class OracleBackend:
    """One process's share computed by the CPU oracle, on torch CPU tensors."""

    def __init__(self, P, x0, nsrc, src_mask, z0, z1, scheme, crit):
        import torch
        self.P = P
        self.scheme = scheme
        self.crit = crit
        n = P.ncell
        self.plane = P.nx * P.ny
        self.x = torch.from_numpy(np.ascontiguousarray(x0, np.float64).ravel().copy())
        self.xh = torch.zeros(n, dtype=torch.float64)
        self.N = {2: [torch.zeros(n, dtype=torch.float64) for _ in range(nsrc)],
                  3: [torch.zeros(n, dtype=torch.float64) for _ in range(nsrc)]}
        self.own = [s for s in range(nsrc) if (src_mask >> s) & 1]
        self.lo, self.hi = z0 * self.plane, z1 * self.plane
        self.t = 0.0
        self.dt = 0.0

    def trace(self, which):
        import torch
        src = self.x if which == 0 else self.xh
        for s in self.own:
            self.N[2 if which == 0 else 3][s][:] = torch.from_numpy(np.ascontiguousarray(self.P.trace(s, src.numpy()).ravel()))

    def _cols(self, kind):
        return np.stack([a.numpy() for a in self.N[kind]])

    def dt_local(self):
        if self.hi <= self.lo:
            return float("inf")
        return self.P.crit_dt_range(self.x.numpy(), self._cols(2), self.lo, self.hi, scheme=self.scheme, **self.crit)

    def _integrate(self, kind, h):
        idx = np.arange(self.lo, self.hi)
        return self.P.integrate_cells(idx, self.x.numpy()[self.lo:self.hi], self._cols(kind), h)

    def step1(self, dt):
        self.dt = dt
        if self.scheme == 3:
            self.xh[self.lo:self.hi] = __import__("torch").from_numpy(self._integrate(2, 0.5 * dt))
        else:
            self.x[self.lo:self.hi] = __import__("torch").from_numpy(self._integrate(2, dt))
            self.t += dt

    def full(self):
        self.x[self.lo:self.hi] = __import__("torch").from_numpy(self._integrate(3, self.dt))
        self.t += self.dt

    def time(self):
        return self.t

    def array(self, kind, source=0):
        return self.x if kind == 0 else (self.xh if kind == 1 else self.N[kind][source])

    def exchanged(self):
        pass


def _worker(rank, world, port, scheme, crit, nsteps, outdir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1201_5651_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _problem()
        P = oracle.Problem.from_workload(w)
        ns = len(w.sources)
        masks = shard.source_masks(ns, world)
        slabs = shard.z_slabs(w.nz, world)
        b = OracleBackend(P, w.x0, ns, masks[rank], *slabs[rank], scheme, crit)
        run = shard.ShardedRun(b, shard.TorchComm("cpu"), ns, w.nz, scheme)
        dts = [run.substep(1e300) for _ in range(nsteps)]
        np.save(os.path.join(outdir, f"x{rank}.npy"), b.x.numpy())
        np.save(os.path.join(outdir, f"dt{rank}.npy"), np.array(dts))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("scheme,crit", [(3, dict(K4=0.25)), (2, dict(K3=0.125))])
def test_two_process_substeps_equal_the_single_process_oracle(tmp_path, scheme, crit):
    import multiprocessing as mp
    import oracle
    nsteps = 3
    ctx = mp.get_context("spawn")
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, scheme, crit, nsteps, str(tmp_path))) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=300)
        assert p.exitcode == 0
    w = _problem()
    P = oracle.Problem.from_workload(w)
    x = np.ascontiguousarray(w.x0.astype(np.float64))
    t = 0.0
    dts = []
    for _ in range(nsteps):
        t_new, dt, _, _ = P.substep(x, t, 1e300, scheme=scheme, **crit)
        dts.append(dt)
        t = t_new
    for r in range(2):
        xr = np.load(tmp_path / f"x{r}.npy")
        assert float(np.max(np.abs(xr - x.ravel()))) <= 1e-13, r
        assert np.allclose(np.load(tmp_path / f"dt{r}.npy"), dts, rtol=1e-14, atol=0), r


def test_partitions_cover_every_source_and_cell_once():
    from paper_1201_5651_gb300 import shard
    for ns, size in [(16, 2), (16, 8), (3, 4), (1, 2)]:
        masks = shard.source_masks(ns, size)
        assert sum(bin(m).count("1") for m in masks) == ns
        assert all((m1 & m2) == 0 for i, m1 in enumerate(masks) for m2 in masks[i + 1:])
        owner = shard.source_owner(ns, size)
        assert all((masks[owner[s]] >> s) & 1 for s in range(ns))
    for nz, size in [(512, 8), (10, 3), (5, 8)]:
        slabs = shard.z_slabs(nz, size)
        assert slabs[0][0] == 0 and slabs[-1][1] == nz
        assert all(a[1] == b[0] for a, b in zip(slabs, slabs[1:]))
        sizes = [b - a for a, b in slabs]
        assert max(sizes) - min(sizes) <= 1
