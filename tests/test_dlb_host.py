"""Host logic of DLB-MPK (Sec. 5, Alg. 2): partition, local problems with halo rows, the
boundary distances I_k, the third-phase schedule and the overhead of Eqs. 10-11; a two-rank
gloo run executes the three phases with numpy row sums and real halo messages."""
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.csgraph as csg

import gen
import oracle
from paper_2405_12525_gb300 import dlb


def _sp(A):
    return sps.csr_matrix((A.val.astype(np.float64), A.col, A.row_ptr), shape=(A.n, A.n))


def _parts(A, parts, balance="nnz"):
    b = dlb.partition_rows(A.n, parts, A.row_ptr if balance == "nnz" else None)
    return b, [dlb.local_problem(A.row_ptr, A.col, A.val, int(b[i]), int(b[i + 1]), b) for i in range(parts)]


def test_partition_rows_balance():
    A = gen.banded_random(5000, stream=31, per_row=9)
    for parts in (1, 2, 3, 7):
        b = dlb.partition_rows(A.n, parts, A.row_ptr)
        assert b[0] == 0 and b[-1] == A.n and np.all(np.diff(b) >= 0) and b.size == parts + 1
        nnz = np.diff(A.row_ptr.astype(np.int64)[b])
        row_max = int(np.diff(A.row_ptr).max())
        assert nnz.max() - A.nnz / parts <= row_max
    b = dlb.partition_rows(10, 4)
    assert list(b) == [0, 2, 5, 8, 10]
    with pytest.raises(ValueError):
        dlb.partition_rows(10, 0)


def test_partitions_without_rows_are_refused():
    # more partitions than rows, or all entries in one row, leave a partition without rows; the
    # emulation refuses that before any device work (no GPU is touched here)
    from paper_2405_12525_gb300.dlb import DlbMpk
    A = gen.laplacian_1d(3)
    with pytest.raises(ValueError, match="owns no row"):
        DlbMpk(A, 5, 2)
    assert list(dlb.partition_rows(3, 5)) == [0, 1, 1, 2, 2, 3]


def test_local_problem_reproduces_global_rows():
    A = gen.banded_random(2000, stream=32, per_row=7, band_frac=0.05)
    x = gen.vector(A.n, stream=33)[:, 0]
    y = _sp(A) @ x
    b, probs = _parts(A, 3)
    for pb in probs:
        n_loc = pb["nl"] + pb["nh"]
        assert pb["halo"].size == pb["nh"] and np.all(np.diff(pb["halo"]) > 0)
        assert np.all((pb["halo"] < pb["r0"]) | (pb["halo"] >= pb["r1"]))
        assert np.all(pb["owner"] == np.searchsorted(b, pb["halo"], side="right") - 1)
        L = sps.csr_matrix((pb["val"], pb["col"], pb["row_ptr"]), shape=(n_loc, n_loc))
        xl = np.concatenate([x[pb["r0"]:pb["r1"]], x[pb["halo"]]])
        yl = L @ xl
        np.testing.assert_allclose(yl[:pb["nl"]], y[pb["r0"]:pb["r1"]], rtol=1e-13, atol=1e-13)
        assert np.all(np.diff(pb["row_ptr"][pb["nl"]:]) == 0)  # halo rows are empty
        # entries kept in stored order: the local column sequence maps back to the global one
        gcol = np.where(pb["col"] < pb["nl"], pb["col"] + pb["r0"],
                        pb["halo"][np.maximum(pb["col"] - pb["nl"], 0)] if pb["nh"] else 0)
        e0, e1 = A.row_ptr[pb["r0"]], A.row_ptr[pb["r1"]]
        assert np.array_equal(gcol, A.col[e0:e1])


def test_send_lists_cover_every_halo():
    A = gen.laplacian_2d(17, 13)
    b, probs = _parts(A, 4)
    sends = dlb.send_lists(probs)
    for i, pb in enumerate(probs):
        got = np.sort(np.concatenate([sends[j][i] for j in sends if i in sends[j]]))
        assert np.array_equal(got, pb["halo"])
    for j, dst in sends.items():
        for i, rows in dst.items():
            assert i != j and np.all((rows >= b[j]) & (rows < b[j + 1]))


def test_boundary_distance_equals_global_graph_distance():
    # symmetric structure: the distance inside the local graph from the halo equals the
    # distance in the whole graph to the nearest row another partition owns
    for A, parts in ((gen.laplacian_2d(12, 9), 3), (gen.laplacian_3d(6, 5, 7), 4), (gen.stencil27(6), 2)):
        G = _sp(A)
        G = (abs(G) + abs(G.T)).tocsr()
        b, probs = _parts(A, parts, balance="rows")
        D = csg.shortest_path(G, unweighted=True)
        for pb in probs:
            outside = np.r_[0:pb["r0"], pb["r1"]:A.n]
            want = D[pb["r0"]:pb["r1"]][:, outside].min(axis=1)
            want = np.where(np.isinf(want), -1, want).astype(np.int64)
            assert np.array_equal(dlb.boundary_distance(pb), want)


def test_boundary_distance_1d_closed_form():
    n = 40
    A = gen.laplacian_1d(n)
    b, probs = _parts(A, 2, balance="rows")
    assert list(b) == [0, 20, 40]
    assert list(dlb.boundary_distance(probs[0])) == list(range(20, 0, -1))
    assert list(dlb.boundary_distance(probs[1])) == list(range(1, 21))


@pytest.mark.parametrize("parts,p_m", [(2, 3), (4, 2), (4, 3), (2, 8)])
def test_overhead_slabs_closed_form(parts, p_m):
    # a 16^3 Laplacian cut into z-slabs of t = 16/parts layers: the rows outside the bulk are
    # those of I_1 .. I_{p_m-1}, p_m-1 layers on each side of a cut, so O_i (Sec. 5, Eq. 2) is
    # (p_m-1)/t for the two end slabs and 2 (p_m-1)/t for inner ones, and the global overhead
    # (Eq. 3) is 2 (parts-1) (p_m-1) / 16
    s = 16
    A = gen.laplacian_3d(s, s, s)
    b, probs = _parts(A, parts, balance="rows")
    t = s // parts
    local, glob = dlb.dlb_overhead(probs, p_m)
    want = [(p_m - 1) / t if i in (0, parts - 1) else 2 * (p_m - 1) / t for i in range(parts)]
    np.testing.assert_allclose(local, want, rtol=0, atol=1e-15)
    assert abs(glob - 2 * (parts - 1) * (p_m - 1) / s) < 1e-15


def test_overhead_without_cut_is_zero():
    A = gen.laplacian_2d(8, 8)
    b, probs = _parts(A, 1)
    assert probs[0]["nh"] == 0
    assert dlb.dlb_overhead(probs, 4) == ([0.0], 0.0)


@pytest.mark.parametrize("num_levels,p_m", [(1, 4), (2, 4), (5, 3), (9, 8), (30, 8), (3, 1)])
def test_phase_iii_schedule_respects_dependencies(num_levels, p_m):
    # have[k] = highest power held by the rows of level k (level 0 = halo).  Phase ii leaves
    # min(k, p_m); every step may only use powers that are already there, and at the end every
    # level holds p_m.  Rows of level k read levels k-1, k, k+1.
    have = [min(k, p_m) for k in range(num_levels)]
    for st in dlb.phase_iii_steps(num_levels, p_m):
        if st[0] == "halo":
            assert have[0] == st[1] - 1
            have[0] = st[1]
            continue
        _, k, q = st
        assert have[k] == q - 1 and have[k - 1] >= q - 1
        if k + 1 < num_levels:
            assert have[k + 1] >= q - 1
        have[k] = q
    assert all(h == p_m for h in have[1:])
    steps = dlb.phase_iii_steps(num_levels, p_m)
    assert sum(1 for s in steps if s[0] == "halo") == p_m - 1


# ----------------------------------------------------------------------------- gloo ranks
def _row_sums(pb, Y, rows, q):
    """Power q of the given local rows from power q-1 (numpy, stored order)."""
    rp, ci, va = pb["row_ptr"], pb["col"], pb["val"].astype(np.float64)
    for r in rows:
        Y[q, r] = np.dot(va[rp[r]:rp[r + 1]], Y[q - 1, ci[rp[r]:rp[r + 1]]])


def _rank_main(rank, world, port, p_m, out):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        A = gen.banded_random(600, stream=34, per_row=6, band_frac=0.02)
        x = gen.vector(A.n, stream=35)[:, 0]
        b = dlb.partition_rows(A.n, world, A.row_ptr)
        probs = [dlb.local_problem(A.row_ptr, A.col, A.val, int(b[i]), int(b[i + 1]), b) for i in range(world)]
        pb = probs[rank]
        sends = dlb.send_lists(probs)
        nl, nh = pb["nl"], pb["nh"]
        Y = np.zeros((p_m + 1, nl + nh))

        def halo(power):
            # owned rows go out along the send lists; halo rows come in from their owners
            reqs = []
            for i, rows in sorted(sends.get(rank, {}).items()):
                reqs.append(dist.isend(torch.from_numpy(Y[power, rows - pb["r0"]].copy()), dst=i))
            for j in np.unique(pb["owner"]):
                sel = np.nonzero(pb["owner"] == j)[0]
                buf = torch.empty(sel.size, dtype=torch.float64)
                dist.recv(buf, src=int(j))
                Y[power, nl + sel] = buf.numpy()
            for r in reqs:
                r.wait()

        Y[0, :nl] = x[pb["r0"]:pb["r1"]]  # phase i
        halo(0)
        d = dlb.boundary_distance(pb)
        cap = np.where(d < 0, p_m, np.minimum(d, p_m))
        level = np.where(d < 0, p_m, d)
        for q in range(1, p_m + 1):  # phase ii
            _row_sums(pb, Y, np.nonzero(cap >= q)[0], q)
        for st in dlb.phase_iii_steps(int(level.max()) + 1 if nl else 1, p_m):  # phase iii
            if st[0] == "halo":
                halo(st[1])
            else:
                _row_sums(pb, Y, np.nonzero(level == st[1])[0], st[2])
        parts = [None] * world
        dist.all_gather_object(parts, Y[:, :nl])
        if rank == 0:
            np.save(out, np.concatenate(parts, axis=1))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,p_m", [(2, 4), (3, 6)])
def test_gloo_ranks_dlb_phases(tmp_path, world, p_m):
    mp = pytest.importorskip("torch.multiprocessing")
    out = str(tmp_path / "y.npy")
    mp.start_processes(_rank_main, args=(world, _free_port(), p_m, out), nprocs=world, start_method="spawn")
    got = np.load(out)
    A = gen.banded_random(600, stream=34, per_row=6, band_frac=0.02)
    x = gen.vector(A.n, stream=35)
    want = oracle.mpk(A, x, p_m)[:, :, 0]
    scale = np.abs(want).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - want) <= 1e-13 * scale)


def test_fig4c_phases_and_order():
    # The 1-D, two-process case of Fig. 4c: the cells phase ii computes (each row of I_k up to
    # power k, the bulk up to p_m), the order of phase iii, and the Lp-diagram order inside
    # phase ii (diagonals of level + power, p ascending, levels counted from the far end)
    from conftest import read_golden
    fig = read_golden("fig4c_dlb_order.txt")
    stage = {(v, p): s for v, p, s in fig}
    p_m = 3
    A = gen.laplacian_1d(8)
    b, probs = _parts(A, 2, balance="rows")
    pb = probs[0]
    assert list(pb["halo"]) == [4]
    d = dlb.boundary_distance(pb)                     # x0..x3 -> 4, 3, 2, 1
    assert list(d) == [4, 3, 2, 1]
    cap = np.minimum(d, p_m)
    phase_ii = {(v, p) for v in range(4) for p in range(1, cap[v] + 1)}
    assert phase_ii == {c for c, s in stage.items() if 1 <= s <= 9}
    # phase iii: ("halo", p) -> vertex 4 at power p; ("rows", k, q) -> the vertex at distance k
    seq = []
    for st in dlb.phase_iii_steps(int(d.max()) + 1, p_m):
        if st[0] == "halo":
            seq.append((4, st[1]))
        else:
            seq += [(int(v), st[2]) for v in np.nonzero(d == st[1])[0]]
    assert seq == sorted((c for c, s in stage.items() if s >= 10), key=lambda c: stage[c])
    # phase ii in the figure follows the Fig. 2 rule on levels counted from x0
    level = d.max() - d
    order = sorted(phase_ii, key=lambda c: (level[c[0]] + c[1], c[1]))
    assert [stage[c] for c in order] == list(range(1, 10))
    assert stage[(4, 0)] == 0


def _failing_rank_main(rank, world, port, out):
    import datetime
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    A = gen.banded_random(300, stream=36, per_row=5, band_frac=0.02)
    b = dlb.partition_rows(A.n, world, A.row_ptr)
    probs = [dlb.local_problem(A.row_ptr, A.col, A.val, int(b[i]), int(b[i + 1]), b) for i in range(world)]
    pb = probs[rank]
    sends = dlb.send_lists(probs)
    peer = 1 - rank
    n_in = int(np.sum(pb["owner"] == peer))
    n_out = int(sends[rank][peer].size)
    # the first exchange completes on both ranks
    w = dist.isend(torch.zeros(n_out, dtype=torch.float64), dst=peer)
    dist.recv(torch.empty(n_in, dtype=torch.float64), src=peer)
    w.wait()
    if rank == 1:
        os._exit(0)  # this rank fails between two exchanges: it never sends again
    # rank 0 learns of it from a bounded wait on the next halo message, not a hang
    try:
        r = dist.irecv(torch.empty(n_in, dtype=torch.float64), src=peer)
        r.wait(timeout=datetime.timedelta(seconds=2))
        result = "no error"
    except Exception as e:  # noqa: BLE001 - any error is the detection
        result = "detected " + type(e).__name__
    with open(out, "w") as f:
        f.write(result)
    os._exit(0)


def test_gloo_rank_failure_is_detected(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    out = str(tmp_path / "result.txt")
    mp.start_processes(_failing_rank_main, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    with open(out) as f:
        assert f.read().startswith("detected")
