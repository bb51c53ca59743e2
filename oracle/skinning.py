"""Skinning and the node graph (Sec. 6.5 initialisation; weights of Eq. 1).

* k-NN: for each query point, the k nodes with the smallest squared distance
  d² = ((dx·dx) + (dy·dy)) + (dz·dz), evaluated in FP32 round-to-nearest on
  the FP32 inputs in exactly that order (the precision the CUDA kernel takes
  the decision in), ties broken by the lower node id.  The result is ordered
  by (d², id), so slot 0 is the nearest node.
* weights: w_k = exp(−‖x − p_k‖² / (2 σ_k²)) (Eq. 1), FP64 from the FP32
  inputs.
* node graph: the 8 nearest other nodes of every node, same rule (Sec. 6.5
  defers the edges to DynamicFusion; k = 8 is the configuration's choice).
"""
import numpy as np

K_SKIN = 4
K_GRAPH = 8


def _d2_fp32(q, p):
    """(nq, np) FP32 squared distances with the fixed operation order."""
    q = q.astype(np.float32)
    p = p.astype(np.float32)
    dx = q[:, None, 0] - p[None, :, 0]
    dy = q[:, None, 1] - p[None, :, 1]
    dz = q[:, None, 2] - p[None, :, 2]
    return ((dx * dx) + (dy * dy)) + (dz * dz)


def knn_fp32(queries, nodes, k, exclude_self=False, chunk=4096):
    """Indices (nq, k) of the k nearest nodes, ordered by (FP32 d², id)."""
    queries = np.asarray(queries, dtype=np.float32)
    nodes = np.asarray(nodes, dtype=np.float32)
    nq, nn = len(queries), len(nodes)
    if nn < k + (1 if exclude_self else 0):
        raise ValueError("not enough nodes for the requested k")
    out = np.empty((nq, k), dtype=np.int64)
    ids = np.arange(nn, dtype=np.uint64)
    for s in range(0, nq, chunk):
        d2 = _d2_fp32(queries[s:s + chunk], nodes)
        if exclude_self:
            rows = np.arange(s, min(s + chunk, nq))
            d2[np.arange(len(rows)), rows] = np.inf
        # d² >= 0, so the IEEE bit pattern orders like the value; append the id
        key = (d2.view(np.uint32).astype(np.uint64) << np.uint64(32)) | ids[None, :]
        part = np.partition(key, k - 1, axis=1)[:, :k]
        part.sort(axis=1)
        out[s:s + chunk] = (part & np.uint64(0xFFFFFFFF)).astype(np.int64)
    return out


def skin_weights(points, node_p, node_sigma, knn):
    """w_k = exp(−‖x − p_k‖² / (2 σ_k²)) in FP64 (Eq. 1)."""
    x = np.asarray(points, dtype=np.float64)
    p = np.asarray(node_p, dtype=np.float64)[knn]
    sig = np.asarray(node_sigma, dtype=np.float64)[knn]
    d2 = np.sum((x[:, None, :] - p) ** 2, axis=-1)
    return np.exp(-d2 / (2.0 * sig * sig))


def skin(surfel_v, node_p, node_sigma, k=K_SKIN):
    knn = knn_fp32(surfel_v, node_p, k)
    return knn, skin_weights(surfel_v, node_p, node_sigma, knn)


def node_graph(node_p, k=K_GRAPH):
    """(Nn, k) neighbour ids of every node, nearest first, self excluded."""
    return knn_fp32(node_p, node_p, k, exclude_self=True)
