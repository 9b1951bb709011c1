"""Host logic of the z-slab decomposition (no GPU).

The library's exchange plan (pure host code) is checked by executing it on a
numpy stand-in of the slabs: after the copies every stored halo plane must
hold the global plane it stands for (wrapped for periodic z), and the planes
beyond a physical z end must be left alone.  The same plan is then executed
between two gloo ranks with point-to-point messages, together with the
max-allreduce of the CFL signal speed, which is how the decomposition maps to
one process per GPU.
"""

import os
import socket
import sys

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hy():
    from paper_1510_05061_gb300 import build, hydro

    build.build()
    hydro.load()
    return hydro


def problem(nz, bcz, n=4):
    p, _ = inputs.rayleigh_taylor(n=n, nz=nz, perturb=False)
    return p.replace(bc_lo=(BC_PERIODIC, BC_PERIODIC, bcz), bc_hi=(BC_PERIODIC, BC_PERIODIC, bcz))


def build_slabs(hy, cp, R, nvar=5, plane=3):
    """Global array g[q, z, c] with distinct values and each rank's copy of
    its planes with NaN halos (stored planes -2 .. nz+1 at index k + 2)."""
    gnz = cp.n[2]
    g = np.arange(nvar * gnz * plane, dtype=np.float64).reshape(nvar, gnz, plane)
    slabs, ext = [], []
    for r in range(R):
        z0, nz = hy.hydro_slab_extent(cp, R, r)
        s = np.full((nvar, nz + 4, plane), np.nan)
        s[:, 2:nz + 2] = g[:, z0:z0 + nz]
        slabs.append(s)
        ext.append((z0, nz))
    return g, slabs, ext


def apply_plan(plan, slabs):
    for src, sp, dst, dp in plan:
        slabs[dst][:, dp + 2:dp + 4] = slabs[src][:, sp + 2:sp + 4]


def check_halos(cp, g, slabs, ext):
    gnz = cp.n[2]
    per = cp.bc_lo[2] == BC_PERIODIC
    R = len(slabs)
    for r, ((z0, nz), s) in enumerate(zip(ext, slabs)):
        for k in (-2, -1, nz, nz + 1):
            gz = z0 + k
            physical = (gz < 0 or gz >= gnz) and not per
            if physical:
                assert np.isnan(s[:, k + 2]).all(), (r, k)
            else:
                np.testing.assert_array_equal(s[:, k + 2], g[:, gz % gnz], err_msg=f"rank {r} plane {k}")


@pytest.mark.parametrize("bcz", [BC_REFLECT, BC_OUTFLOW, BC_PERIODIC])
@pytest.mark.parametrize("nz,R", [(8, 1), (8, 2), (9, 2), (13, 4), (12, 3), (8, 4), (11, 5)])
def test_plan_fills_every_halo(hy, nz, R, bcz):
    cp = hy.make_problem(problem(nz, bcz))
    ext = [hy.hydro_slab_extent(cp, R, r) for r in range(R)]
    # contiguous cover of [0, nz), sizes differ by at most one, larger first
    assert ext[0][0] == 0 and sum(e[1] for e in ext) == nz
    assert all(ext[i][0] + ext[i][1] == ext[i + 1][0] for i in range(R - 1))
    assert max(e[1] for e in ext) - min(e[1] for e in ext) <= 1
    assert [e[1] for e in ext] == sorted((e[1] for e in ext), reverse=True)
    plan = hy.hydro_slabs_exchange_plan(cp, R)
    per = bcz == BC_PERIODIC
    assert len(plan) == (2 * R if per else 2 * (R - 1))
    g, slabs, ext = build_slabs(hy, cp, R)
    apply_plan(plan, slabs)
    check_halos(cp, g, slabs, ext)


def test_invalid_decompositions(hy):
    cp = hy.make_problem(problem(8, BC_REFLECT))
    for R in (0, -1, 5, 9):
        assert hy.load().hydro_slab_state_bytes(cp, R, 0) == 0
        assert hy.load().hydro_slabs_exchange_plan(cp, R, None, 0) == hy.HYDRO_ERR_INVALID_ARG
    assert hy.load().hydro_slab_state_bytes(cp, 2, 2) == 0
    z0, nz = hy.hydro_slab_extent(cp, 4, 3)
    assert (z0, nz) == (6, 2)
    # one state buffer: 5 variables x (nz + 4) planes x 4 x 4 cells x 8 bytes
    assert hy.load().hydro_slab_state_bytes(cp, 4, 3) == 5 * 6 * 16 * 8
    p2, _ = inputs.sod(n=16, ndim=2)
    assert hy.load().hydro_slab_state_bytes(hy.make_problem(p2), 1, 0) == 0


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nz, bcz, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1510_05061_gb300 import hydro as hy

    dist.init_process_group("gloo", rank=rank, world_size=world)
    cp = hy.make_problem(problem(nz, bcz))
    g, slabs, ext = build_slabs(hy, cp, world)
    mine = torch.from_numpy(slabs[rank].copy())
    # each rank sends and receives the copies that involve it, over gloo
    ops = []
    for src, sp, dst, dp in hy.hydro_slabs_exchange_plan(cp, world):
        if src == rank and dst == rank:
            mine[:, dp + 2:dp + 4] = mine[:, sp + 2:sp + 4].clone()
        elif src == rank:
            ops.append(dist.P2POp(dist.isend, mine[:, sp + 2:sp + 4].contiguous(), dst))
        elif dst == rank:
            buf = torch.empty_like(mine[:, dp + 2:dp + 4])
            ops.append((dist.P2POp(dist.irecv, buf, src), dp, buf))
    reqs = dist.batch_isend_irecv([o if isinstance(o, dist.P2POp) else o[0] for o in ops]) if ops else []
    for q in reqs:
        q.wait()
    for o in ops:
        if not isinstance(o, dist.P2POp):
            _, dp, buf = o
            mine[:, dp + 2:dp + 4] = buf
    # the dt reduction: max of the ranks' signal speeds
    speed = torch.tensor([1.0 + 0.25 * rank], dtype=torch.float64)
    dist.all_reduce(speed, op=dist.ReduceOp.MAX)
    np.save(os.path.join(outdir, f"slab{rank}.npy"), mine.numpy())
    with open(os.path.join(outdir, f"speed{rank}.txt"), "w") as fh:
        fh.write(repr(float(speed)))
    dist.destroy_process_group()


@pytest.mark.parametrize("nz,bcz", [(9, BC_REFLECT), (8, BC_PERIODIC)])
def test_exchange_between_gloo_ranks(hy, tmp_path, nz, bcz):
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_rank, args=(world, free_port(), nz, bcz, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    cp = hy.make_problem(problem(nz, bcz))
    g, _, ext = build_slabs(hy, cp, world)
    slabs = [np.load(tmp_path / f"slab{r}.npy") for r in range(world)]
    check_halos(cp, g, slabs, ext)
    for r in range(world):
        assert float((tmp_path / f"speed{r}.txt").read_text()) == 1.25
