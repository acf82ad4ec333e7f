"""The sharded form of the update on CPU ranks: slabs along z, one layer of
post-collision populations exchanged with each neighbour per step (the overlap
communicator of the guide's section "Communication"), checked bit for bit
against the single-domain oracle.  Ranks are gloo processes on the host; each
steps its slab with the oracle's collision and streaming.  A rank whose halo
message never arrives gets a timeout error instead of hanging.

The shipped GPU path runs one lattice per GPU (replicas only); this test covers
the exchange logic of the decomposition the design describes for several GPUs.
"""
import datetime
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(kind):
    from paper_2307_11752_gb300 import inputs as I

    if kind == "cavity":
        m = I.cavity_box(9, 8, 10)
        wu = np.zeros((256, 3))
        wu[I.LID] = (0.05, 0.0, 0.01)
        return dict(material=m, periodic=0, tau=0.57, wall_u=wu, force=(0.0, 0.0, 0.0), gamma=None,
                    noise=I.population_noise(5, 19, m, 1e-4))
    m = I.channel(8, 7, 12)
    m[:, :, :] = I.FLUID  # periodic box with a porous field and a force
    return dict(material=m, periodic=7, tau=0.7, wall_u=np.zeros((256, 3)), force=(2e-5, 0.0, -1e-5),
                gamma=I.smoothed_porosity(6, m), noise=I.population_noise(7, 19, m, 1e-3))


def _lattice(oracle, c, material, periodic, gamma):
    return oracle.Lattice(oracle.D3Q19, material, c["tau"], periodic=periodic, force=c["force"],
                          gamma=gamma, wall_u=c["wall_u"])


def _worker(rank, world, port, kind, steps, drop_at, results):
    import torch
    import torch.distributed as dist

    from oracle import oracle
    from paper_2307_11752_gb300 import inputs as I

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=4))
    c = _case(kind)
    m = c["material"]
    nz = m.shape[0]
    z0, z1 = rank * nz // world, (rank + 1) * nz // world
    zper = bool(c["periodic"] & 4)
    full = _lattice(oracle, c, m, c["periodic"], c["gamma"])
    f = np.ascontiguousarray(full.init_equilibrium(*I.rest(m.shape)) + c["noise"])
    own = np.ascontiguousarray(f[:, z0:z1])
    lo_peer = rank - 1 if rank > 0 else (world - 1 if zper else None)
    hi_peer = rank + 1 if rank < world - 1 else (0 if zper else None)
    void = np.zeros((1,) + m.shape[1:], np.uint8)
    ext_mat = np.concatenate([m[[(z0 - 1) % nz]] if lo_peer is not None else void, m[z0:z1],
                              m[[z1 % nz]] if hi_peer is not None else void])
    g = c["gamma"]
    mine = _lattice(oracle, c, m[z0:z1], c["periodic"] & 3, None if g is None else g[z0:z1])
    ext = _lattice(oracle, c, ext_mat, c["periodic"] & 3, None)
    status = "ok"
    try:
        for s in range(steps):
            post = mine.collide(own)
            halo_lo = torch.zeros(post[:, :1].shape, dtype=torch.float64)
            halo_hi = torch.zeros_like(halo_lo)
            reqs = []
            skip = drop_at is not None and rank == 1 and s == drop_at
            if lo_peer is not None:
                if not skip:
                    reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(post[:, :1])), lo_peer, tag=2 * s))
                reqs.append(dist.irecv(halo_lo, lo_peer, tag=2 * s + 1))
            if hi_peer is not None:
                if not skip:
                    reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(post[:, -1:])), hi_peer, tag=2 * s + 1))
                reqs.append(dist.irecv(halo_hi, hi_peer, tag=2 * s))
            if skip:
                status = "dropped"
                break
            for r in reqs:
                r.wait()
            e = np.ascontiguousarray(np.concatenate([halo_lo.numpy(), post, halo_hi.numpy()], axis=1))
            pre = np.ascontiguousarray(np.concatenate([np.zeros_like(post[:, :1]), own, np.zeros_like(post[:, :1])], axis=1))
            own = np.ascontiguousarray(ext.stream(e, pre)[:, 1:-1])
    except RuntimeError as err:  # gloo timeout of a halo message that never came
        status = "timeout: " + str(err).splitlines()[0][:80]
    results[rank] = (status, own if status == "ok" else None, z0, z1)
    if status == "ok":
        dist.barrier()
        dist.destroy_process_group()


def _run(kind, steps, drop_at=None):
    import torch.multiprocessing as mp

    world = 2
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), kind, steps, drop_at, results), nprocs=world,
                       join=True, start_method="spawn")
    return dict(results)


@pytest.mark.parametrize("kind", ["cavity", "porous_periodic"])
def test_slab_decomposition_is_bit_identical(oracle, kind):
    from paper_2307_11752_gb300 import inputs as I

    steps = 12
    res = _run(kind, steps)
    c = _case(kind)
    m = c["material"]
    full = _lattice(oracle, c, m, c["periodic"], c["gamma"])
    f = np.ascontiguousarray(full.init_equilibrium(*I.rest(m.shape)) + c["noise"])
    full.step(f, steps)
    fl = m == I.FLUID
    for rank, (status, own, z0, z1) in res.items():
        assert status == "ok"
        assert np.array_equal(own[:, fl[z0:z1]], f[:, z0:z1][:, fl[z0:z1]])


def test_missing_halo_message_times_out(oracle):
    res = _run("cavity", 6, drop_at=3)
    assert res[1][0] == "dropped"
    assert res[0][0].startswith("timeout")
