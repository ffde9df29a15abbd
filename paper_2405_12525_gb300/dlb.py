"""DLB-MPK (Sec. 5, Alg. 2) with the partitions of a row-wise distributed matrix held on one
device, plus the host logic shared with a multi-process setting.

Each partition i owns a contiguous range of rows.  Its local problem is square: the owned rows
(columns relabelled, entries in stored order) followed by one empty row per halo vertex (a
remote row it reads).  The BFS levels of the local problem are built from the halo rows as
level 0, so level k is the paper's I_k, the rows k steps from the boundary, and the rows at
level >= p_m form the bulk M.  The three phases:
  i)   the initial halo exchange: the halo rows receive x;
  ii)  one level-blocked launch in which a row of level L takes powers 1..min(L, p_m)
       (plan option level_capped);
  iii) for p = 1..p_m-1: the halo rows receive power p of their owners' rows, then the rows
       of levels k = 1..p_m-p advance from power k+p-1 to k+p, k ascending (one SpMV over
       each level's rows).
Every row sum keeps its stored order, so the result equals the single-matrix MPK bit for bit.
The halo exchange between partitions is a device gather here (on several GPUs it would be a
peer copy or NCCL send/recv of the same rows); TRAD (p_m halo exchanges, each followed by a
full local SpMV) runs on the same data for comparison.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------- host logic
def partition_rows(n: int, parts: int, row_ptr=None):
    """Bounds of `parts` contiguous row ranges, balanced by stored entries when row_ptr is
    given, else by rows."""
    if parts < 1:
        raise ValueError("parts >= 1")
    if row_ptr is None:
        return np.linspace(0, n, parts + 1).round().astype(np.int64)
    rp = np.asarray(row_ptr, dtype=np.int64)
    targets = np.linspace(0, rp[-1], parts + 1)
    b = np.searchsorted(rp, targets).astype(np.int64)
    b[0], b[-1] = 0, n
    return np.maximum.accumulate(b)


def local_problem(row_ptr, col, val, r0: int, r1: int, bounds):
    """Local square problem of the rows [r0, r1): owned rows first (columns relabelled, entries
    in stored order), then one empty row per halo vertex (sorted global ids).  Returns a dict
    with the local CSR, the halo ids and their owning partitions."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col, dtype=np.int64)
    e0, e1 = rp[r0], rp[r1]
    cols = ci[e0:e1]
    outside = (cols < r0) | (cols >= r1)
    halo = np.unique(cols[outside])
    nl, nh = r1 - r0, halo.size
    lc = np.where(outside, nl + np.searchsorted(halo, cols), cols - r0)
    lrp = np.concatenate([rp[r0:r1 + 1] - e0, np.full(nh, e1 - e0)])
    owner = np.searchsorted(np.asarray(bounds), halo, side="right") - 1
    return {"r0": int(r0), "r1": int(r1), "nl": int(nl), "nh": int(nh), "halo": halo, "owner": owner,
            "row_ptr": lrp.astype(np.int32), "col": lc.astype(np.int32),
            "val": np.asarray(val)[e0:e1]}


def send_lists(problems):
    """For every partition j and every requester i: the global rows j sends to i."""
    sends = {}
    for i, pb in enumerate(problems):
        for j in np.unique(pb["owner"]):
            sends.setdefault(int(j), {})[i] = pb["halo"][pb["owner"] == j]
    return sends


def boundary_distance(pb):
    """Distance of every local row from the halo (the levels of the local problem from the
    halo rows; -1 for rows that cannot reach the halo), computed on the host."""
    import scipy.sparse as sps
    n = pb["nl"] + pb["nh"]
    A = sps.csr_matrix((np.ones(pb["col"].size), pb["col"], pb["row_ptr"]), shape=(n, n))
    G = (A + A.T).tocsr()
    d = np.full(n, -1, dtype=np.int64)
    front = np.arange(pb["nl"], n)
    d[front] = 0
    k = 0
    while front.size:
        k += 1
        nb = np.unique(G[front].indices)
        front = nb[d[nb] < 0]
        d[front] = k
    return d[:pb["nl"]]


def phase_iii_steps(num_levels: int, p_m: int):
    """Steps of the third phase for a partition whose local levels run 0..num_levels-1 (level 0
    the halo): ("halo", p) brings power p of the halo rows, ("rows", k, q) computes power q of
    the rows of level k from their power q-1.  Round p (1 <= p < p_m) advances the levels
    k = 1..p_m-p, in ascending order, from power k+p-1 to k+p."""
    steps = []
    for p in range(1, p_m):
        steps.append(("halo", p))
        for k in range(1, p_m - p + 1):
            if k < num_levels:
                steps.append(("rows", k, k + p))
    return steps


def dlb_overhead(problems, p_m: int):
    """Local overheads O_i = 1 - |M_i| / N_i,r (Sec. 5, Eq. 2) and the global overhead (Eq. 3):
    the share of owned rows closer than p_m to the boundary."""
    local = []
    for pb in problems:
        d = boundary_distance(pb)
        bulk = int(np.sum((d >= p_m) | (d < 0)))
        local.append(1.0 - bulk / pb["nl"] if pb["nl"] else 0.0)
    rows = np.array([pb["nl"] for pb in problems], dtype=np.float64)
    return local, float(np.sum(rows * np.array(local)) / max(1.0, rows.sum()))


def mpi_overhead(problems):
    """Halo rows over all partitions divided by the total number of rows (the communication
    overhead of Sec. 4, Eq. 1): the same for TRAD and DLB-MPK."""
    return sum(pb["nh"] for pb in problems) / max(1, sum(pb["nl"] for pb in problems))


# ----------------------------------------------------------------------------- device emulation
class DlbMpk:
    """All partitions of A on the current device.

    The local vectors of all partitions live in one buffer: partition i holds its powers
    0..p_m as a block of (p_m+1) x n_loc,i x m doubles in its plan's row order (halo rows
    first), so a halo exchange is one indexed row copy for all partitions and a per-level
    step is one multi-segment SpMV launch for all partitions, as if the processes ran
    concurrently.  run() / trad() act on the resident local vectors (the distributed setting:
    x and the powers stay with their owners); apply() adds the scatter of X into the local
    vectors and the gather of the powers into A's own numbering."""

    def __init__(self, A, parts: int, p_m: int, nrhs: int = 1, cache_bytes: int = 0, value_type=None,
                 balance: str = "nnz", engine: int = 0):
        import torch
        from . import MAX_ROW_SEGMENTS, MPK_F64, ORDER_PLAN, CsrMatrix, build_levels, build_levels_from, plan
        if parts > MAX_ROW_SEGMENTS:
            raise ValueError(f"at most {MAX_ROW_SEGMENTS} partitions")
        self.torch = torch
        self.n, self.p_m, self.m = A.n, p_m, nrhs
        self.bounds = partition_rows(A.n, parts, A.row_ptr if balance == "nnz" else None)
        empty = np.nonzero(np.diff(self.bounds) == 0)[0]
        if empty.size:  # a process of Alg. 2 owns at least one row
            raise ValueError(f"partition {int(empty[0])} of {parts} owns no row of the {A.n}: use fewer partitions")
        self.problems = [local_problem(A.row_ptr, A.col, A.val, int(self.bounds[i]), int(self.bounds[i + 1]), self.bounds)
                         for i in range(parts)]
        vt = MPK_F64 if value_type is None else value_type
        dt = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[vt]
        n_loc = [pb["nl"] + pb["nh"] for pb in self.problems]
        self.row0 = np.concatenate([[0], np.cumsum([(p_m + 1) * nl for nl in n_loc])]).astype(np.int64)
        self.Y_all = torch.empty((int(self.row0[-1]), nrhs), dtype=torch.float64, device="cuda")
        self.parts = []
        for i, pb in enumerate(self.problems):
            dA = CsrMatrix(torch.from_numpy(pb["row_ptr"]).cuda(), torch.from_numpy(pb["col"]).cuda(),
                           torch.as_tensor(pb["val"], dtype=torch.float64).to(dt).cuda(), False)
            if pb["nh"]:
                L = build_levels_from(dA, np.arange(pb["nl"], n_loc[i]))
            else:
                L = build_levels(dA, 0)
            P = plan(dA, L, p_max=p_m, nrhs=nrhs, order=ORDER_PLAN, cache_bytes=cache_bytes,
                     level_capped=bool(pb["nh"]), engine=engine)
            lp = L.level_ptr.cpu().numpy().astype(np.int64)
            perm = L.perm.cpu().numpy().astype(np.int64)
            iperm = L.iperm.cpu().numpy().astype(np.int64)
            if pb["nh"] and (lp[1] != pb["nh"] or not np.array_equal(perm[:pb["nh"]], np.arange(pb["nl"], n_loc[i]))):
                raise RuntimeError("level 0 must be exactly the halo rows, in ascending order")
            Y = self.Y_all[int(self.row0[i]):int(self.row0[i + 1])].view(p_m + 1, n_loc[i], nrhs)
            self.parts.append({"pb": pb, "A": dA, "L": L, "P": P, "lp": lp, "iperm": iperm, "Y": Y})

        def row_of(i, k, r):  # row of Y_all holding power k of plan row r of partition i
            return self.row0[i] + k * n_loc[i] + r

        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int64)).cuda()
        # exchange of power k: the halo rows of every partition (sorted global ids, plan rows
        # [0, nh)) receive power k of their owners' rows
        src0, dst0 = [], []
        for i, part in enumerate(self.parts):
            pb = part["pb"]
            for j in np.unique(pb["owner"]):
                sel = np.nonzero(pb["owner"] == j)[0]
                own = self.parts[j]
                src0.append(row_of(j, 0, own["iperm"][pb["halo"][sel] - own["pb"]["r0"]]))
                dst0.append(row_of(i, 0, sel))
        src0 = np.concatenate(src0) if src0 else np.zeros(0, np.int64)
        dst0 = np.concatenate(dst0) if dst0 else np.zeros(0, np.int64)
        owner_of = np.searchsorted(self.row0, src0, side="right") - 1
        dest_of = np.searchsorted(self.row0, dst0, side="right") - 1
        nl_arr = np.array(n_loc, dtype=np.int64)
        self.halo_idx = [(dev(src0 + k * nl_arr[owner_of]), dev(dst0 + k * nl_arr[dest_of])) for k in range(p_m)]
        self.halo_rows = int(src0.size)
        # load / store between A's numbering and the local vectors (owned rows only)
        g_src, l_dst = [], []
        for i, part in enumerate(self.parts):
            pb = part["pb"]
            g_src.append(np.arange(pb["r0"], pb["r1"]))
            l_dst.append(row_of(i, 0, part["iperm"][:pb["nl"]]))
        g_src, l_dst = np.concatenate(g_src), np.concatenate(l_dst)
        self.load_idx = (dev(g_src), dev(l_dst))
        dest_part = np.searchsorted(self.row0, l_dst, side="right") - 1
        self.store_idx = [(dev(l_dst + k * nl_arr[dest_part]), dev(g_src + k * A.n)) for k in range(p_m + 1)]
        self.steps = phase_iii_steps(max(p["lp"].size - 1 for p in self.parts), p_m)
        self.overhead_local, self.overhead = dlb_overhead(self.problems, p_m)

    def _halo(self, k: int):
        from . import copy_rows
        src, dst = self.halo_idx[k]
        copy_rows(self.Y_all, src, self.Y_all, dst)

    def _rows(self, ranges, q: int):
        """Power q of the given plan-row ranges (one per partition) from power q-1."""
        from . import spmv_rows_multi
        seg = [(part, lo, hi) for part, (lo, hi) in zip(self.parts, ranges) if hi > lo]
        if seg:
            spmv_rows_multi([s[0]["P"] for s in seg], [s[1] for s in seg], [s[2] for s in seg],
                            [s[0]["Y"][q - 1] for s in seg], [s[0]["Y"][q] for s in seg])

    def load(self, X):
        """Owned rows of every partition's power 0 <- X (A's numbering, n x m)."""
        from . import copy_rows
        copy_rows(X, self.load_idx[0], self.Y_all, self.load_idx[1])

    def store(self, Y):
        """Y[k] (A's numbering) <- power k of every partition's owned rows."""
        from . import copy_rows
        Yf = Y.view(-1, self.m)
        for src, dst in self.store_idx:
            copy_rows(self.Y_all, src, Yf, dst)

    def run(self):
        """DLB-MPK on the resident local vectors (Alg. 2): phase i, the level-capped launches
        of phase ii, and the p_m-1 rounds of phase iii."""
        self._halo(0)
        for part in self.parts:
            part["P"].apply(part["Y"][0], self.p_m, Y=part["Y"])
        for step in self.steps:
            if step[0] == "halo":
                self._halo(step[1])
                continue
            _, k, q = step
            self._rows([(int(p["lp"][k]), int(p["lp"][k + 1])) if p["pb"]["nh"] and k + 1 < p["lp"].size else (0, 0)
                        for p in self.parts], q)

    def run_trad(self):
        """TRAD (Alg. 1) on the resident local vectors: p_m times a halo exchange of the last
        power and one SpMV over every partition's owned rows."""
        for q in range(1, self.p_m + 1):
            self._halo(q - 1)
            self._rows([(p["pb"]["nh"], p["pb"]["nh"] + p["pb"]["nl"]) for p in self.parts], q)

    def apply(self, X, Y=None, trad: bool = False):
        """Y[k] = A^k X for k = 0..p_m (X, Y in A's own numbering)."""
        if Y is None:
            Y = self.torch.empty((self.p_m + 1, self.n, self.m), dtype=self.torch.float64, device="cuda")
        self.load(X)
        self.run_trad() if trad else self.run()
        self.store(Y)
        return Y

    def trad(self, X, Y=None):
        return self.apply(X, Y, trad=True)
