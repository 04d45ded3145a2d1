"""Multi-rank host logic on CPU: world-size-2 gloo process groups.

* Sharding: every unit lands on exactly one rank, contiguous, balanced.
* Forward: emitters split by slices, each rank computes its own slab; the
  concatenated slabs equal the unsharded batch (no collective on this path).
* Adjoint of one pupil with its planes split over ranks: the all-reduced
  partial gradients equal the unsharded gradient (the one real exchange).
* The step time reported by a multi-rank run is the maximum over ranks.
The arithmetic on each rank is the FP64 oracle; what is tested is the
partitioning and the collective around it."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import adjoint as oadj
from oracle import bessel as ob
from oracle.optics import Optics
from paper_2502_03170_gb300 import shard
from paper_2502_03170_gb300 import workloads as W

WORLD = 2


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_split_even_covers_units():
    for n in (0, 1, 5, 128, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard.split_even(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges[:-1], ranges[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.split_even(4, 2, 2)


def test_split_weighted_balances_slices():
    c = W.bessel()
    offs = c["z_offsets"]
    total = int(offs[-1])
    for world in (1, 2, 4, 8):
        ranges = [shard.split_weighted(offs, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == len(offs) - 1
        for (a, b), (c2, d) in zip(ranges[:-1], ranges[1:]):
            assert b == c2
        per = [int(offs[b]) - int(offs[a]) for a, b in ranges]
        assert sum(per) == total
        assert max(per) - min(per) <= 2 * 64          # within two emitters' stacks
    # degenerate: more ranks than emitters, empty emitters
    offs = np.array([0, 0, 3, 3, 4])
    ranges = [shard.split_weighted(offs, r, 8) for r in range(8)]
    assert ranges[0][0] == 0 and ranges[-1][1] == 4
    assert sum(int(offs[b]) - int(offs[a]) for a, b in ranges) == 4


def _init(rank, port):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port,
                            rank=rank, world_size=WORLD)


def _rank_adjoint(rank, port, out_dir, case):
    _init(rank, port)
    try:
        opt, n_pupil, grid, zern, pm, T = case
        lo, hi = shard.split_even(len(grid["z"]), rank, WORLD)
        g = dict(grid, z=grid["z"][lo:hi])
        L, gW, gc, _ = oadj.loss_and_grad(opt, n_pupil, g, zern, pm, T[lo:hi])
        t = torch.tensor(np.concatenate([[L], gW.ravel(), gc]), dtype=torch.float64)
        shard.allreduce_sum_(t)
        t_max = shard.max_over_ranks([1.0 + rank, 5.0 - rank])
        np.save(os.path.join(out_dir, "r%d.npy" % rank), t.numpy())
        np.save(os.path.join(out_dir, "m%d.npy" % rank), np.array(t_max))
    finally:
        dist.destroy_process_group()


def _rank_forward(rank, port, out_dir, case):
    _init(rank, port)
    try:
        opt, depth, zern, offs, z, geo = case
        e0, e1 = shard.split_weighted(offs, rank, WORLD)
        lo_offs, lz = shard.local_batch(offs, z, e0, e1)
        I = ob.psf_bessel_batch(opt, depth[e0:e1], zern[e0:e1], lo_offs, lz, project=True,
                                **geo)
        np.save(os.path.join(out_dir, "f%d.npy" % rank), I)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_adjoint_allreduce_gloo():
    g = np.random.default_rng(3)
    d = W.optics_gibson_lanni(1.0)
    opt = Optics.from_dict(d)
    n_pupil = 24
    grid = dict(nx=12, ny=10, dx=0.04, dy=0.04, z=np.linspace(-0.6, 0.6, 5))
    zern = np.zeros(11)
    zern[3:11] = g.normal(0, 0.1, 8)
    pm = 0.1 * g.normal(size=(n_pupil, n_pupil))
    T = np.abs(g.normal(size=(5, 12, 10))) * 1e-3
    L, gW, gc, _ = oadj.loss_and_grad(opt, n_pupil, grid, zern, pm, T)
    with tempfile.TemporaryDirectory() as tmp:
        mp.spawn(_rank_adjoint, args=(free_port(), tmp, (opt, n_pupil, grid, zern, pm, T)),
                 nprocs=WORLD, join=True)
        r0 = np.load(os.path.join(tmp, "r0.npy"))
        r1 = np.load(os.path.join(tmp, "r1.npy"))
        m0 = np.load(os.path.join(tmp, "m0.npy"))
    assert np.array_equal(r0, r1)                     # every rank holds the sum
    full = np.concatenate([[L], gW.ravel(), gc])
    assert np.allclose(r0, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    assert list(m0) == [2.0, 5.0]                     # max over ranks


def test_sharded_bessel_forward_gloo():
    c = W.bessel(n_emitters=7, n_theta=24, n_r=32, nx=10, nz_lo=1, nz_hi=4)
    opt = Optics.from_dict(c["optics"])
    geo = dict(n_theta=24, n_r=32, nx=10, ny=10, dx=c["dx"], dy=c["dy"])
    full = ob.psf_bessel_batch(opt, c["depth"], c["zernike"], c["z_offsets"], c["z"],
                               project=True, **geo)
    with tempfile.TemporaryDirectory() as tmp:
        mp.spawn(_rank_forward,
                 args=(free_port(), tmp, (opt, c["depth"], c["zernike"], c["z_offsets"],
                                          c["z"], geo)),
                 nprocs=WORLD, join=True)
        parts = [np.load(os.path.join(tmp, "f%d.npy" % r)) for r in range(WORLD)]
    assert np.array_equal(np.concatenate(parts, axis=0), full)
