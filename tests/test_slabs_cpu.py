"""Row-slab decomposition on CPU: the partition, the populations that cross
a slab boundary, and the whole exchange protocol run by two gloo ranks.

Each rank owns a band of rows of a periodic lattice plus one ghost row on
either side; a step collides its rows (the FP64 oracle's collision, which
is local to a node), sends its edge rows' crossing populations to its
neighbours (slabs.CROSS_UP upwards, slabs.CROSS_DOWN downwards, along
slabs.exchange_schedule) and pull-streams from the extended band.  After
many steps the gathered bands must equal the oracle's run of the whole
lattice bit for bit: streaming only moves values, and the collision of a
node does not depend on which band holds it.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_crossing_populations_follow_the_lattice_velocities(orc):
    from paper_2602_14667_gb300 import slabs
    cx, cy, w, ex, ey, psi = orc.lattice()
    cy_all = list(cy) + [int(e) for e in ey for _ in range(2)]
    assert slabs.CROSS_UP == tuple(p for p in range(19) if cy_all[p] == 1)
    assert slabs.CROSS_DOWN == tuple(p for p in range(19) if cy_all[p] == -1)
    assert len(slabs.CROSS_UP) == len(slabs.CROSS_DOWN) == 5     # 3 f + one g vector each way


def test_partition_tiles_the_rows_and_the_schedule_closes_the_ring():
    from paper_2602_14667_gb300 import slabs
    for ny, k in ((10, 3), (64, 2), (7, 7), (5, 1)):
        r = slabs.partition(ny, k)
        assert r[0][0] == 0 and r[-1][1] == ny and all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
        sch = slabs.exchange_schedule(k)
        assert sorted(lo for lo, _ in sch) == list(range(k)) and all(up == (lo + 1) % k for lo, up in sch)
    with pytest.raises(ValueError):
        slabs.partition(3, 4)


def test_combine_totals_weights_means_and_rms_by_nodes():
    from paper_2602_14667_gb300 import slabs
    a = dict(mass=10.0, mom_x=1.0, mom_y=2.0, bsum_x=0.5, bsum_y=0.25, e_kin=1.0, e_mag=2.0, cross_hel=3.0,
             divb_max=0.1, jz_max=0.2, omega_max=0.3, divb_rms=1.0, step=7)
    b = dict(mass=30.0, mom_x=-1.0, mom_y=1.0, bsum_x=0.5, bsum_y=0.75, e_kin=3.0, e_mag=0.0, cross_hel=-1.0,
             divb_max=0.4, jz_max=0.1, omega_max=0.2, divb_rms=2.0, step=7)
    t = slabs.combine_totals([(a, 1), (b, 3)], nx=4)
    assert t["mass"] == 40.0 and t["mom_x"] == 0.0 and t["bsum_y"] == 1.0
    assert t["e_kin"] == (1.0 * 1 + 3.0 * 3) / 4 and t["cross_hel"] == (3.0 - 3.0) / 4
    assert t["divb_max"] == 0.4 and t["jz_max"] == 0.2 and t["omega_max"] == 0.3
    assert abs(t["divb_rms"] - np.sqrt((1.0 * 1 + 4.0 * 3) / 4)) < 1e-15 and t["step"] == 7
    tw = slabs.combine_totals([(a, 1), (b, 3)], nx=4, wall_x=True)      # valid columns 2 of 4: same weights
    assert abs(tw["divb_rms"] - t["divb_rms"]) < 1e-15


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


NX, NY, STEPS, TAU = 12, 10, 25, (0.56, 0.62)
CX = np.array([0, -1, -1, -1, 0, 1, 1, 1, 0])
EX = np.array([0, -1, 0, 1, 0])


def _global_state(orc):
    rng = np.random.default_rng(5)
    p = orc.Params(NX, NY, *TAU)
    f, g = orc.init(p, *(rng.uniform(-0.05, 0.05, (NY, NX)) for _ in range(4)),
                    rho=rng.uniform(0.97, 1.03, (NY, NX)))
    return p, f, g


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2602_14667_gb300 import slabs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.build()
    _, f, g = _global_state(oracle)
    y0, y1 = slabs.partition(NY, world)[rank]
    h = y1 - y0
    pl = oracle.Params(NX, h, *TAU)
    # this rank's pre-collision band as 19 planes
    band = np.concatenate([f[:, y0:y1], g[:, :, y0:y1].reshape(10, h, NX)])
    below = [lo for lo, up in slabs.exchange_schedule(world) if up == rank][0]
    above = [up for lo, up in slabs.exchange_schedule(world) if lo == rank][0]
    for _ in range(STEPS):
        fs, gs = oracle.collide(pl, np.ascontiguousarray(band[:9]), np.ascontiguousarray(band[9:].reshape(5, 2, h, NX)))
        post = np.zeros((19, h + 2, NX))
        post[:9, 1:-1] = fs
        post[9:, 1:-1] = gs.reshape(10, h, NX)
        # the exchange: my top row's upward populations to the slab above,
        # my bottom row's downward ones to the slab below (gloo: send then
        # receive, ranks ordered so that the pairs never both wait)
        up_send = torch.from_numpy(post[list(slabs.CROSS_UP), h].copy())
        dn_send = torch.from_numpy(post[list(slabs.CROSS_DOWN), 1].copy())
        up_recv = torch.empty_like(up_send)
        dn_recv = torch.empty_like(dn_send)
        reqs = [dist.isend(up_send, above, tag=1), dist.isend(dn_send, below, tag=2),
                dist.irecv(up_recv, below, tag=1), dist.irecv(dn_recv, above, tag=2)]
        for r in reqs:
            r.wait()
        post[list(slabs.CROSS_UP), 0] = up_recv.numpy()      # ghost row below
        post[list(slabs.CROSS_DOWN), h + 1] = dn_recv.numpy()  # ghost row above
        # pull streaming from the extended band (x periodic)
        cyv = np.array(slabs.CY)
        cxv = np.concatenate([CX, np.repeat(EX, 2)])
        for p in range(19):
            src = post[p, 1 - cyv[p]:h + 1 - cyv[p]]
            band[p] = np.roll(src, cxv[p], axis=1)
    got = [torch.zeros((19, hh, NX), dtype=torch.float64) for hh in
           (b - a for a, b in slabs.partition(NY, world))] if rank == 0 else None
    if rank == 0:
        got[0] = torch.from_numpy(band)
        for r in range(1, world):
            dist.recv(got[r], r)
        out["bands"] = [t.numpy() for t in got]
    else:
        dist.send(torch.from_numpy(band), 0)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_whole_lattice_bitwise(orc):
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        bands = out["bands"]
    p, f, g = _global_state(orc)
    f, g = orc.run(p, f, g, STEPS)
    whole = np.concatenate([f, g.reshape(10, NY, NX)])
    assert np.array_equal(np.concatenate(bands, axis=1), whole)


_PARTS = (dict(mass=10.0, mom_x=1.0, mom_y=2.0, bsum_x=0.5, bsum_y=0.25, e_kin=1.0, e_mag=2.0, cross_hel=3.0,
               divb_max=0.1, jz_max=0.2, omega_max=0.3, divb_rms=1.0, step=7),
          dict(mass=30.0, mom_x=-1.0, mom_y=1.0, bsum_x=0.5, bsum_y=0.75, e_kin=3.0, e_mag=0.0, cross_hel=-1.0,
               divb_max=0.4, jz_max=0.1, omega_max=0.2, divb_rms=2.0, step=7))
_ROWS = (1, 3)


def _totals_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2602_14667_gb300 import slabs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    for wall_x in (False, True):
        t = slabs.allreduce_totals(_PARTS[rank], _ROWS[rank], nx=4, wall_x=wall_x)
        out[(rank, wall_x)] = t
    dist.barrier()
    dist.destroy_process_group()


def test_allreduce_totals_on_two_gloo_ranks_equals_combine_totals():
    """One slab per rank: the two FP64 all-reduces give every rank the
    totals combine_totals forms from all the slabs' totals."""
    from paper_2602_14667_gb300 import slabs
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_totals_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        got = dict(out)
    for wall_x in (False, True):
        want = slabs.combine_totals(list(zip(_PARTS, _ROWS)), nx=4, wall_x=wall_x)
        for r in range(world):
            t = got[(r, wall_x)]
            assert set(t) == set(want)
            for k, v in want.items():
                assert abs(t[k] - v) <= 1e-15 * max(1.0, abs(v)), (r, wall_x, k, t[k], v)
