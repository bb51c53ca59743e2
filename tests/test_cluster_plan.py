"""Host logic of the cluster PCG's launch plan (no GPU): the plan built by
the library for an upper 6x6 block pattern is checked table by table, and
the symmetric SpMV that the cluster kernel performs from it -- u pushed by
each row's owner into the halos that need it, every home block's A_ij u_j
for its row and, off the diagonal, its A_ijᵀ u_i sent to a receive slot of
the column's owner -- is replayed in numpy with the kernel's index
arithmetic and must equal the product with the whole symmetric matrix."""
import numpy as np
import pytest

import synth
import paper_1904_13073_gb300 as sw
from oracle import skinning as OSKIN
from oracle import solver as OS

GROUPS = 96            # row groups of a CTA (768 threads, 8 lanes each)
SMEM_LIMIT = 230_000   # about the opt-in shared memory of a CTA on this part


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1904_13073_gb300 import build as B
    B.build()


def upper_pattern(scene, n_sample=None, seed=0):
    """(row_ptr, col) of the library's upper block layout: skinning pairs of
    the surfels (a sample of them for large scenes), the node graph and the
    diagonal; every row leads with its diagonal block."""
    v = scene.surfel_v
    if n_sample is not None and n_sample < len(v):
        v = v[np.random.default_rng(seed).choice(len(v), n_sample, replace=False)]
    knn = OSKIN.knn_fp32(v.astype(np.float32), scene.node_p.astype(np.float32), 4)
    graph = OSKIN.node_graph(scene.node_p.astype(np.float32))
    n = len(scene.node_p)
    keys = OS.BlockMatrix.pattern(n, knn, graph).keys
    r, c = keys // n, keys % n
    up = r <= c
    r, c = r[up], c[up]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, r + 1, 1)
    return np.cumsum(row_ptr).astype(np.int32), c.astype(np.int32)


def node4(scene):
    out = np.zeros((len(scene.node_p), 4), np.float32)
    out[:, :3] = scene.node_p
    return out


def unpack(plan):
    C, NR, NB, NG, n, NH, NP = (int(x) for x in plan[:7])
    o = 7
    rb = plan[o:o + C + 1]; o += C + 1
    bb = plan[o:o + C + 1]; o += C + 1
    gb = plan[o:o + C + 1]; o += C + 1
    pb = plan[o:o + C + 1]; o += C + 1
    rows = plan[o:o + n]; o += n
    hb = plan[o:o + n + C]; o += n + C
    go = plan[o:o + n + C]; o += n + C
    po = plan[o:o + n + C]; o += n + C
    nnzb = int(bb[C])
    blk = plan[o:o + nnzb]; o += nnzb
    col = plan[o:o + nnzb]; o += nnzb
    o2t = plan[o:o + nnzb]; o += nnzb
    push = plan[o:o + int(pb[C])]; o += int(pb[C])
    assert o == len(plan)
    return dict(C=C, NR=NR, NB=NB, NG=NG, n=n, NH=NH, NP=NP, rb=rb, bb=bb, gb=gb, pb=pb, rows=rows, hb=hb, go=go,
                po=po, blk=blk, col=col, o2t=o2t, push=push)


def replay_spmv(P, row_ptr, colidx, A, u):
    """The cluster kernel's symmetric SpMV from the plan's tables: the u
    pushes fill every CTA's halo, each home block adds A_ij u_j to its row
    and sends A_ijᵀ u_i to a receive slot of row j's owner, and every row
    adds its receive slots."""
    C, n = P["C"], P["n"]

    def cta(c):
        r0, nr = int(P["rb"][c]), int(P["rb"][c + 1] - P["rb"][c])
        sl = slice(r0 + c, r0 + c + nr + 1)
        return nr, P["rows"][r0:r0 + nr], P["hb"][sl], P["go"][sl], P["po"][sl]
    # each CTA's u slots: own rows, then halo slots filled by the owners' pushes
    slot_row = [dict() for _ in range(C)]
    U = [dict() for _ in range(C)]
    for c in range(C):
        nr, rows, _, _, po = cta(c)
        assert nr <= P["NR"]
        for a, i in enumerate(rows):
            slot_row[c][a] = int(i)
            U[c][a] = u[i]
            for x in range(po[a], po[a + 1]):
                tg = int(P["push"][P["pb"][c] + x])
                peer, slot = tg >> 16, tg & 0xffff
                assert peer != c and slot >= P["rb"][peer + 1] - P["rb"][peer] and slot not in U[peer]
                slot_row[peer][slot] = int(i)
                U[peer][slot] = u[i]
    for c in range(C):
        nr = int(P["rb"][c + 1] - P["rb"][c])
        assert len(U[c]) - nr <= P["NH"]
    w = np.zeros((n, 6))
    recv = [dict() for _ in range(C)]
    for c in range(C):
        nr, rows, hb, _, _ = cta(c)
        assert int(P["bb"][c + 1] - P["bb"][c]) == hb[nr] <= P["NB"]
        for a, i in enumerate(rows):
            for e in range(hb[a], hb[a + 1]):
                k = int(P["bb"][c]) + e
                b, ci, tg = int(P["blk"][k]), int(P["col"][k]), int(P["o2t"][k])
                assert slot_row[c][ci] == colidx[b] and row_ptr[i] <= b < row_ptr[i + 1]
                w[i] += A[b] @ U[c][ci]
                if e == hb[a]:
                    assert colidx[b] == i and tg == -1          # the diagonal block leads its row
                else:
                    owner, slot = tg >> 16, tg & 0xffff
                    assert slot not in recv[owner]
                    recv[owner][slot] = (int(colidx[b]), A[b].T @ u[i])
    for c in range(C):
        nr, rows, _, go, _ = cta(c)
        assert int(P["gb"][c + 1] - P["gb"][c]) == go[nr] <= P["NG"]
        assert sorted(recv[c]) == list(range(int(go[nr])))  # every slot filled once
        for a, j in enumerate(rows):
            for x in range(go[a], go[a + 1]):
                row, v = recv[c][x]
                assert row == j
                w[j] += v
    return w


def symmetric_product(row_ptr, colidx, A, u):
    n = len(row_ptr) - 1
    w = np.zeros((n, 6))
    for i in range(n):
        for b in range(row_ptr[i], row_ptr[i + 1]):
            j = colidx[b]
            w[i] += A[b] @ u[j]
            if j != i:
                w[j] += A[b].T @ u[i]
    return w


@pytest.mark.parametrize("which", ["tiny", "mid", "full"])
def test_cluster_plan_tables_and_replayed_spmv(which):
    if which == "tiny":
        scene, sample = synth.plain_tiny(seed=0), None
    elif which == "mid":
        scene, sample = synth.random_scene(seed=5, n_surfels=20000, n_nodes=600), None
    else:
        scene, sample = synth.plain_full(seed=0), 40000     # 2048 nodes
    row_ptr, colidx = upper_pattern(scene, sample)
    n = len(row_ptr) - 1
    plan, smem = sw.sw_debug_cluster_plan(16, row_ptr, colidx, node4(scene), SMEM_LIMIT)
    P = unpack(plan)
    assert P["C"] == 16 and P["n"] == n and smem <= SMEM_LIMIT
    # every node is a row of exactly one CTA, within the rows two groups serve
    assert sorted(P["rows"].tolist()) == list(range(n))
    assert P["NR"] <= 2 * GROUPS and P["NR"] == int(np.max(np.diff(P["rb"])))
    # every block is the home block of exactly one CTA, CTA-major and row by row
    assert sorted(P["blk"].tolist()) == list(range(int(row_ptr[-1])))
    assert P["NB"] == int(np.max(np.diff(P["bb"]))) and P["NG"] == int(np.max(np.diff(P["gb"])))
    assert int(P["gb"][-1]) == int(row_ptr[-1]) - n       # one receive slot per off-diagonal block
    rng = np.random.default_rng(1)
    A = rng.standard_normal((int(row_ptr[-1]), 6, 6))
    u = rng.standard_normal((n, 6))
    np.testing.assert_allclose(replay_spmv(P, row_ptr, colidx, A, u), symmetric_product(row_ptr, colidx, A, u),
                               rtol=1e-12, atol=1e-12)


def test_cluster_plan_refuses_what_does_not_fit():
    scene = synth.plain_full(seed=0)
    row_ptr, colidx = upper_pattern(scene, 40000)
    with pytest.raises(sw.SwError):
        sw.sw_debug_cluster_plan(16, row_ptr, colidx, node4(scene), 100_000)   # too little shared memory
    with pytest.raises(sw.SwError):
        sw.sw_debug_cluster_plan(2, row_ptr, colidx, node4(scene), 10 ** 9)    # 1024 rows for one CTA
    bad = colidx.copy()
    bad[row_ptr[3]] = 4                                                      # row 3 without its diagonal first
    with pytest.raises(sw.SwError):
        sw.sw_debug_cluster_plan(16, row_ptr, bad, node4(scene), SMEM_LIMIT)
