"""Host logic of the partitioned solve on CPU: the parts' local meshes, the
ghost plan, and the halo exchange on gloo ranks (one rank per part) driving
the oracle's operator and predictor.  The owned results must equal the
unpartitioned oracle's."""
import os
import socket
import sys

import numpy as np
import pytest

import synth
import oracle
from paper_1805_03981_gb300 import partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _curved(N, k, seed, periodic):
    rng = np.random.default_rng(seed)
    fr = synth.mesh.random_frames(N ** 3, rng)
    mesh = synth.cube_mesh(N, q=k, periodic=periodic, deform=synth.mesh.curving(0.05), frames=fr)
    x = synth.solution_node_positions(mesh, k)
    rho, c = synth.fields.cfg2_coefficients(x)
    return mesh, rho, c, synth.configs.random_state(N ** 3, k, seed + 1)


@pytest.mark.parametrize("P", [2, 3, 5])
@pytest.mark.parametrize("periodic", [True, False])
def test_split_meshes_and_ghost_plan(P, periodic):
    mesh, rho, c, _ = _curved(3, 2, 7, periodic)
    parts = partition.split(mesh, P, rho, c)
    owned_all = np.concatenate([p["owned"] for p in parts])
    assert np.array_equal(np.sort(owned_all), np.arange(mesh["n_elem"]))
    for q, part in enumerate(parts):
        lm, no = part["mesh"], part["owned"].size
        elems = np.concatenate([part["owned"], part["ghost"]])
        nbr, nbf, ori = lm["nbr"], lm["nbr_face"], lm["orient"]
        # connectivity is reciprocal with the same face and orientation codes
        for e in range(lm["n_elem"]):
            for f in range(6):
                en = nbr[e, f]
                if en < 0:
                    continue
                assert nbr[en, nbf[e, f]] == e and nbf[en, nbf[e, f]] == f
                assert elems[en] == mesh["nbr"][elems[e], f]
                assert ori[e, f] == mesh["orient"][elems[e], f]
        # owned elements keep every face of the whole mesh
        assert np.array_equal(nbr[:no] >= 0, np.asarray(mesh["nbr"])[part["owned"]] >= 0)
        # every ghost comes from an owned element of another part
        for g, sp, se in zip(part["ghost"], part["src_part"], part["src_elem"]):
            assert sp != q and parts[sp]["owned"][se] == g
        assert np.array_equal(lm["nodes"], np.asarray(mesh["nodes"])[elems])
    sends, recvs = partition.send_lists(parts), partition.recv_slots(parts)
    for p in range(P):
        for q in range(P):
            assert sends[p][q].size == recvs[q][p].size


def _local_state(part, U_global):
    return np.concatenate([U_global[part["owned"]], U_global[part["ghost"]]])


def test_part_operator_equals_whole_operator():
    """With ghosts copied from their owners, each part's operator on its
    owned elements equals the whole mesh's (same formulas per element)."""
    k = 2
    mesh, rho, c, U = _curved(3, k, 11, False)
    whole = oracle.Oracle(mesh, k, rho, c).apply(U)
    for P in (2, 4):
        for part in partition.split(mesh, P, rho, c):
            o = oracle.Oracle(part["mesh"], k, part["rho"], part["c"])
            R = o.apply(_local_state(part, U))[: part["owned"].size]
            ref = whole[part["owned"]]
            assert np.abs(R - ref).max() <= 1e-13 * np.abs(whole).max()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _exchange(dist, torch, parts, me, Uloc, sends, recvs):
    """Refresh this rank's ghost tiles from their owners (point to point)."""
    P = len(parts)
    no = parts[me]["owned"].size
    reqs = []
    bufs = {}
    for q in range(P):
        if q != me and sends[me][q].size:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(Uloc[sends[me][q]])), dst=q))
        if q != me and recvs[me][q].size:
            bufs[q] = torch.empty((recvs[me][q].size,) + Uloc.shape[1:], dtype=torch.float64)
            reqs.append(dist.irecv(bufs[q], src=q))
    for r in reqs:
        r.wait()
    for q, b in bufs.items():
        Uloc[no + recvs[me][q]] = b.numpy()


def _rank(rank, world, port, qout):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    k = 2
    mesh, rho, c, U = _curved(3, k, 21, True)
    parts = partition.split(mesh, world, rho, c)
    sends, recvs = partition.send_lists(parts), partition.recv_slots(parts)
    part = parts[rank]
    no = part["owned"].size
    o = oracle.Oracle(part["mesh"], k, part["rho"], part["c"])
    Uloc = np.zeros((part["mesh"]["n_elem"],) + U.shape[1:])
    Uloc[:no] = U[part["owned"]]                  # a rank knows only what it owns
    dt = 0.01
    for _ in range(2):                            # two ADER steps: one exchange each
        Ubar = o.tck(Uloc, dt, 2)
        _exchange(dist, torch, parts, rank, Ubar, sends, recvs)
        Uloc = Uloc + o.apply(Ubar)
    dist.barrier()
    dist.destroy_process_group()
    qout.put((rank, part["owned"], Uloc[:no]))


def test_halo_exchange_on_gloo_ranks_matches_whole_oracle():
    import torch.multiprocessing as mp
    k = 2
    mesh, rho, c, U = _curved(3, k, 21, True)
    ref = oracle.Oracle(mesh, k, rho, c).ader(U, 0.01, 2, 2)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.empty_like(ref)
    for _, owned, Uo in out:
        got[owned] = Uo
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
