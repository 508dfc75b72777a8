"""One mesh over several ranks, on the CPU: the slab partition, the halo lists
(dgm_partition_slabs, dgm_halo_build through the binding) and the per-stage
halo exchange (Halo.exchange) with two gloo ranks.  Each rank evaluates the
oracle's right-hand side on its owned elements from its local state (owned
coefficients plus ghosts received from the other rank) and steps LSRK4 stage
by stage with an exchange after each stage; both must reproduce the
single-domain oracle on the owned elements.  No GPU: the coefficient packing
here is a numpy gather of the same lists the device pack kernel uses."""
import os
import socket
import sys

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


def test_slabs_are_balanced_and_ordered(D):
    xyz, tets = W.kuhn_mesh(4, jitter=0.1, seed=5)
    for nparts in (1, 2, 3, 5):
        part = D.partition_slabs(xyz, tets, nparts, axis=2)
        counts = np.bincount(part, minlength=nparts)
        assert counts.max() - counts.min() <= 1 and counts.sum() == len(tets)
        z = W.centroids(xyz, tets)[:, 2]
        for r in range(nparts - 1):
            assert z[part == r].max() <= z[part == r + 1].min()
    with pytest.raises(D.DgmError):
        D.partition_slabs(xyz, tets, 0)
    with pytest.raises(D.DgmError):
        D.partition_slabs(xyz, tets, 2, axis=3)


def _face_neighbours(tets):
    faces = {}
    for e, t in enumerate(np.sort(tets, axis=1)):
        for f in range(4):
            key = tuple(np.delete(t, f))
            faces.setdefault(key, []).append(e)
    nb = [set() for _ in range(len(tets))]
    for es in faces.values():
        if len(es) == 2:
            nb[es[0]].add(es[1])
            nb[es[1]].add(es[0])
    return nb


@pytest.mark.parametrize("nparts", [2, 3])
def test_halo_lists_match_between_peers(D, nparts):
    xyz, tets = W.kuhn_mesh(3, jitter=0.1, seed=6)
    part = D.partition_slabs(xyz, tets, nparts, axis=2)
    halos = [D.Halo(tets, part, nparts, r) for r in range(nparts)]
    nb = _face_neighbours(tets)
    for r, h in enumerate(halos):
        l2g = h.local_to_global
        owned = l2g[:h.n_owned]
        assert np.array_equal(owned, np.nonzero(part == r)[0])
        want_ghosts = sorted({n for e in owned for n in nb[e] if part[n] != r})
        assert list(l2g[h.n_owned:]) == want_ghosts
        assert set(h.peers) == {int(part[g]) for g in want_ghosts}
        for q, peer in enumerate(h.peers):
            other = halos[peer]
            qq = list(other.peers).index(r)
            sent = l2g[h.send[q]]
            got = other.local_to_global[other.recv[qq]]
            assert np.array_equal(sent, got)           # entry by entry
            assert np.all(part[sent] == r) and np.all(sent[:-1] < sent[1:])
            assert np.all(h.send[q] < h.n_owned) and np.all(other.recv[qq] >= other.n_owned)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
    import workloads as W
    from oracle_ref import build
    from oracle.solver import LSRK4_A, LSRK4_B, LSRK4_C
    from paper_2002_08733_gb300 import dgmax as D
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        xyz, tets = W.kuhn_mesh(3, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=7)
        K, p, S = len(tets), 2, 2
        eps = W.lognormal_material(K, 2.0, 0.3, 8)
        pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=10.0, order=2)
        dt = W.stable_dt(2 / 3, p)
        part = D.partition_slabs(xyz, tets, world, axis=2)
        h = D.Halo(tets, part, world, rank)
        l2g, n = h.local_to_global, h.n_owned
        u = W.random_state(K, S, p, seed=9)
        aux = W.random_state(K, S, p, seed=10) * 0.1
        # single-domain oracle (every rank computes it) and this rank's local one
        glob = build(xyz, tets, p, eps, 1.0, "upwind", pml=pml, S=S)
        loc = build(xyz, tets[l2g], p, eps[l2g], 1.0, "upwind", pml=pml, S=S,
                    rows=np.arange(n))
        ul = np.full_like(u[l2g], np.nan)              # ghosts unknown until exchanged
        ul[:n] = u[l2g[:n]]
        al = aux[l2g].copy()

        def refresh(state):
            h.exchange(pack=lambda q: torch.from_numpy(np.ascontiguousarray(state[h.send[q]])),
                       unpack=lambda q, b: state.__setitem__(h.recv[q], b.numpy()),
                       isend=lambda b, peer: dist.isend(b, peer),
                       irecv=lambda b, peer: dist.irecv(b, peer),
                       empty_like_recv=lambda q: torch.empty((len(h.recv[q]),) + state.shape[1:],
                                                             dtype=torch.float64))

        refresh(ul)
        assert np.isfinite(ul).all()
        ref, ref_aux = glob.unpack(glob.rhs(glob.pack(u, aux), 0.3))
        got, got_aux = loc.unpack(loc.rhs(loc.pack(ul, al), 0.3), nelem=n)
        err_rhs = float(np.abs(got - ref[l2g[:n]]).max() / np.abs(ref).max())
        err_aux = float(np.abs(got_aux - ref_aux[l2g[:n]]).max() / np.abs(ref_aux).max())
        # three LSRK4 steps, stage by stage, halo refreshed after every stage
        x_ref = glob.lsrk4(glob.pack(u, aux), 0.0, dt, 3)
        res_u, res_a = np.zeros_like(ul[:n]), np.zeros_like(al[:n])
        t = 0.0
        for _ in range(3):
            for k in range(5):
                du, da = loc.unpack(loc.rhs(loc.pack(ul, al), t + LSRK4_C[k] * dt), nelem=n)
                res_u = LSRK4_A[k] * res_u + dt * du
                res_a = LSRK4_A[k] * res_a + dt * da
                ul[:n] += LSRK4_B[k] * res_u
                al[:n] += LSRK4_B[k] * res_a
                refresh(ul)
            t += dt
        u_ref, _ = glob.unpack(x_ref)
        err_step = float(np.abs(ul[:n] - u_ref[l2g[:n]]).max() / np.abs(u_ref).max())
        out.put((rank, err_rhs, err_aux, err_step, n, len(l2g) - n))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_single_domain(D):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=600)
        assert pr.exitcode == 0
    res = [q.get(timeout=5) for _ in range(2)]
    assert sum(r[4] for r in res) == 162
    for rank, e_rhs, e_aux, e_step, n_owned, n_ghost in res:
        assert n_ghost > 0
        assert e_rhs < 1e-13 and e_aux < 1e-13 and e_step < 1e-12, (rank, e_rhs, e_aux, e_step)
