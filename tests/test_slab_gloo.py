"""Slab decomposition of the particle system over several ranks (gloo on
host cores, world sizes 2 and 4) against the single-domain FP64 oracle: the
forces of every owned particle -- Eq. 1 plasma and wall DPD, Eq. 3
interface, Eq. 2 LJ, bonds and angles, Eq. 4 Morse, the body force -- agree
to 1e-12 relative; every particle is owned exactly once before and after a
migration; FP64 sums of the kinetic energy and momentum equal the
single-domain sums."""
import os
import socket

import numpy as np
import pytest


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def system(seed=61):
    """A walled 24 x 10 x 8 channel at rho = 3 with three 300-particle
    platelets, two of them within Morse reach of each other across the
    middle of the channel, the third near the periodic x face; shells
    jittered so that bonds and angles carry load."""
    import synth
    s = synth.platelet_system((24.0, 10.0, 8.0), 3 * 24 * 10 * 8, 3, 300, synth.scaled_radii(300), walls=True,
                              body_force=0.02, seed=seed,
                              centers=[(10.6, 5.0, 4.0), (13.4, 5.2, 4.1), (23.2, 5.0, 4.0)])
    rng = np.random.default_rng(seed)
    plt = s.tag >= 0
    s.x[plt] += 0.02 * rng.standard_normal((int(plt.sum()), 3))
    s.x[:, 0] %= s.box[0]
    return s


def _rank(rank, world, port, out_q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        from paper_2205_14121_gb300 import slab
        s = system()
        p = O.system_params(s)
        pb = O.system_params(s, lj_eps=0.0, m_D=0.0, f_A=0.0, a_ff=0.0, a_fw=0.0, a_fp=0.0, gamma=0.0, sigma=0.0)
        S = slab.Slabs(s.box, rank, world)
        me = slab.SlabSystem.scatter(S, s.x, s.v, s.tag, s.X0)
        bonds_by_id = s.bonds
        angles_by_id = s.angles
        theta0 = s.theta0
        n_time = 3

        def pair_force(x, v, tag, ids, X0, pairs):
            return O.pair_forces(p, x, v, tag.astype(np.int32), pairs, X0=X0, ids=ids.astype(np.int32),
                                 n_time=n_time)

        def bonded_force(ids, x):
            # bonds and angles of the owned platelets, over the owned arrays
            pos = -np.ones(s.n, np.int64)
            pos[ids] = np.arange(len(ids))
            bm = (pos[bonds_by_id[:, 0]] >= 0) & (pos[bonds_by_id[:, 1]] >= 0)
            am = np.all(pos[angles_by_id] >= 0, axis=1)
            O.set_angles(pb, pos[angles_by_id[am]], theta0[am])
            f, _ = O.forces_brute(pb, x, np.zeros_like(x), s.tag[ids], bonds=pos[bonds_by_id[bm]],
                                  r0=s.r0[bm], level_mask=O.LVL_PLT)
            return f

        def reach_pair(ta, tb):
            return np.where((ta >= 0) & (tb >= 0), slab.REACH_PLT, slab.REACH_FLUID)

        f = me.forces(pair_force, bonded_force, reach_pair, body_force=s.body_force)
        ref, _ = O.forces_brute(p, s.x, s.v, s.tag, X0=s.X0, bonds=s.bonds, r0=s.r0, n_time=n_time)
        err = np.abs(f - ref[me.id]).max() / np.abs(ref).max()
        ke = me.reduce_fp64([0.5 * (me.v[me.tag != -2] ** 2).sum()])[0]
        mom = me.reduce_fp64(me.v[me.tag != -2].sum(0))
        ids_before = me.id.copy()
        # move everything by a third of a slab along x and migrate
        me.x[:, 0] = (me.x[:, 0] + s.box[0] / world / 3.0) % s.box[0]
        me.migrate()
        out_q.put((rank, float(err), len(ids_before), ids_before.tolist(), me.id.tolist(), float(ke),
                   mom.tolist(), bool(np.all(S.owners(me.x, me.tag) == rank))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_slab_decomposition_matches_single_domain_oracle(world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    s = system()
    res.sort()
    for r in res:
        assert r[1] < 1e-12, f"rank {r[0]}: relative force error {r[1]}"
        assert r[7], "a migrated particle is not owned by the rank that holds it"
    before = np.concatenate([r[3] for r in res])
    after = np.concatenate([r[4] for r in res])
    assert np.array_equal(np.sort(before), np.arange(s.n))
    assert np.array_equal(np.sort(after), np.arange(s.n))
    assert all(r[2] > 0 for r in res)
    mob = s.tag != -2
    assert res[0][5] == pytest.approx(0.5 * (s.v[mob] ** 2).sum(), rel=1e-13)
    assert np.allclose(res[0][6], s.v[mob].sum(0), rtol=0, atol=1e-9)
