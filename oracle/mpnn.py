"""Plain FP64 reference of the learned warm start (test infrastructure only:
the tests and the benchmark use it; the CUDA library never does).

The componentwise method solves every SCC C of a level by the power series
P_0 = W_C, P_{k+1} = c A_C^T P_k (Sec. 4.3.2), W being the inflow-adjusted
weight of Eq. (PR:levels).  A warm start replaces the first term by a guess
R0 and continues the series from the residual of the guess; this module is
the definition of the guess the GPU computes: a two-layer message-passing
network over the SCC's internal in-edges, evaluated here in float64 with the
same bf16-rounded weights.

The solution is R_C = W_C + M_C W_C with M_C = (I - c A_C^T)^-1 - I >= 0, so
R_i - W_i is about b_i mean_C(W) when W does not vary much inside C, b_i
being the amplification of row i (the row sum of M_C, weighted by W).  The
network guesses b_i from the structure alone, so that it can run once per
graph before the level loop, and the solver forms the guess from the W of
the level when it gets there (and a guess depends on the graph and the
network only, so it serves every solve of the partition).  Per SCC vertex i
of component C (internal in-degree d_i >= 1, internal out-degree o_i,
external in-degree e_i):
  x_i  = [log1p(d_i), log1p(outdeg_i), log|C|, o_i / outdeg_i, log1p(e_i),
          log1p(outdeg_i - o_i), 1, 0]
  m_i  = mean of x_j over the internal in-edges j -> i
  h_i  = relu(A1 x_i + B1 m_i + b1)                       (64)
  m'_i = mean of h_j over the internal in-edges j -> i
  g_i  = relu(A2 h_i + B2 m'_i + b2)                      (64)
  yhat = v . g_i + b3
target y_i = log(max((R_i - W_i) / mean_C(W), 1e-6)) for the solved R
(components with mean_C(W) = 0 are left out); loss = mean (yhat_i - y_i)^2.
The guess is R0_i = W_i + exp(clamp(yhat_i, -14, 9)) mean_C(W).

Parameters, one float32 vector: A1[64][8], B1[64][8], b1[64], A2[64][64],
B2[64][64], b2[64], v[64], b3[1] (row-major, output index first).
"""
from __future__ import annotations

import numpy as np

F0 = 8
H = 64
SHAPES = [("A1", (H, F0)), ("B1", (H, F0)), ("b1", (H,)), ("A2", (H, H)), ("B2", (H, H)), ("b2", (H,)),
          ("v", (H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
YHAT_MIN, YHAT_MAX = -14.0, 9.0
B_FLOOR = 1e-6


def unpack(theta):
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def bf16_round(a):
    """float32 -> nearest bfloat16 (ties to even), returned as float32.
    The IEEE binary32 pattern keeps its top 16 bits after adding half an
    ulp of bfloat16 plus the tie-breaking parity bit."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def features(rowptr, col, part, c, u, R):
    """Inputs of the network for every SCC vertex of a solved graph.

    Returns (rows, X, in_ptr, in_src, y, mask): rows are the SCC vertices in
    ascending id; in_ptr/in_src list, per row, the row indices of its
    internal in-neighbours (same component, self-loops dropped); W is formed
    from R as in Eq. (PR:levels) (for the target only: the inputs do not
    depend on R)."""
    rowptr = np.asarray(rowptr, np.int64)
    col = np.asarray(col, np.int64)
    n = rowptr.shape[0] - 1
    src = np.repeat(np.arange(n), np.diff(rowptr))
    keep = src != col
    src, dst = src[keep], col[keep]
    outdeg = np.bincount(src, minlength=n).astype(np.float64)
    comp = np.asarray(part.comp, np.int64)
    ctype = np.zeros(part.n_comp, np.int64)
    ctype[comp] = part.type
    size = np.bincount(comp, minlength=part.n_comp)
    R = np.asarray(R, np.float64)
    z = np.where(outdeg > 0, R / np.maximum(outdeg, 1), 0.0)
    ext = comp[src] != comp[dst]
    W = np.asarray(u, np.float64).copy()
    np.add.at(W, dst[ext], c * z[src[ext]])
    is_scc = ctype[comp] == 1
    rows = np.nonzero(is_scc)[0]
    ridx = -np.ones(n, np.int64)
    ridx[rows] = np.arange(rows.size)
    inte = (~ext) & is_scc[dst]
    order = np.lexsort((src[inte], dst[inte]))
    e_src, e_dst = src[inte][order], dst[inte][order]
    din = np.bincount(ridx[e_dst], minlength=rows.size)
    dout = np.bincount(ridx[e_src], minlength=rows.size)
    ein = np.bincount(dst[ext], minlength=n)
    in_ptr = np.concatenate([[0], np.cumsum(din)])
    in_src = ridx[e_src]
    X = np.zeros((rows.size, F0))
    X[:, 0] = np.log1p(din)
    X[:, 1] = np.log1p(outdeg[rows])
    X[:, 2] = np.log(size[comp[rows]])
    X[:, 3] = dout / np.maximum(outdeg[rows], 1)
    X[:, 4] = np.log1p(ein[rows])
    X[:, 5] = np.log1p(outdeg[rows] - dout)
    X[:, 6] = 1.0
    cmean = component_means(comp, part.n_comp, W)
    mw = cmean[comp[rows]]
    mask = mw > 0
    b = np.where(mask, (R[rows] - W[rows]) / np.where(mask, mw, 1.0), 1.0)
    y = np.where(mask, np.log(np.maximum(b, B_FLOOR)), 0.0)
    return rows, X, in_ptr, in_src, y, mask


def component_means(comp, n_comp, W):
    """mean_C(W) per component C."""
    comp = np.asarray(comp, np.int64)
    s = np.zeros(n_comp)
    np.add.at(s, comp, W)
    return s / np.maximum(np.bincount(comp, minlength=n_comp), 1)


def guess(yhat, W_rows, mean_rows):
    """R0 of the SCC rows from the network's yhat and the level's W."""
    return W_rows + np.exp(np.clip(yhat, YHAT_MIN, YHAT_MAX)) * mean_rows


def _mean_in(in_ptr, in_src, Hm):
    d = np.diff(in_ptr)
    seg = np.repeat(np.arange(d.size), d)
    out = np.zeros((d.size, Hm.shape[1]))
    np.add.at(out, seg, Hm[in_src])
    return out / np.maximum(d, 1)[:, None]


def forward(theta, X, in_ptr, in_src):
    """yhat and the intermediates; theta is used as given (round it first)."""
    p = unpack(theta)
    m = _mean_in(in_ptr, in_src, X)
    z1 = X @ p["A1"].T + m @ p["B1"].T + p["b1"]
    h = np.maximum(z1, 0.0)
    m2 = _mean_in(in_ptr, in_src, h)
    z2 = h @ p["A2"].T + m2 @ p["B2"].T + p["b2"]
    g = np.maximum(z2, 0.0)
    yhat = g @ p["v"] + p["b3"][0]
    return yhat, dict(m=m, z1=z1, h=h, m2=m2, z2=z2, g=g)


def loss(theta, X, in_ptr, in_src, y, mask):
    yhat, _ = forward(theta, X, in_ptr, in_src)
    d = (yhat - y)[mask]
    return float(np.mean(d * d)) if d.size else 0.0


def loss_and_grad(theta, X, in_ptr, in_src, y, mask):
    """Analytic gradient of the mean squared error (backward pass written
    out layer by layer: head, layer 2, mean aggregation, layer 1)."""
    p = unpack(theta)
    yhat, t = forward(theta, X, in_ptr, in_src)
    N = max(int(mask.sum()), 1)
    r = np.where(mask, yhat - y, 0.0)
    L = float(np.sum(r * r) / N)
    dy = 2.0 * r / N
    gr = {}
    gr["v"] = t["g"].T @ dy
    gr["b3"] = np.array([dy.sum()])
    dz2 = np.outer(dy, p["v"]) * (t["z2"] > 0)
    gr["A2"] = dz2.T @ t["h"]
    gr["B2"] = dz2.T @ t["m2"]
    gr["b2"] = dz2.sum(axis=0)
    dh = dz2 @ p["A2"]
    dm2 = dz2 @ p["B2"]
    d = np.diff(in_ptr)
    seg = np.repeat(np.arange(d.size), d)
    np.add.at(dh, in_src, dm2[seg] / np.maximum(d, 1)[seg, None])
    dz1 = dh * (t["z1"] > 0)
    gr["A1"] = dz1.T @ X
    gr["B1"] = dz1.T @ t["m"]
    gr["b1"] = dz1.sum(axis=0)
    return L, pack(gr)


def init_params(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases except
    b3 = 1 (a guess of R = e W before any training); numpy's generator.
    Only a starting point for tests; the library draws its own."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SHAPES:
        if name.startswith("b"):
            d[name] = np.zeros(shape)
        else:
            fan_in = shape[1] if len(shape) == 2 else shape[0]
            d[name] = rng.uniform(-1, 1, shape) / np.sqrt(fan_in)
    d["b3"] = np.array([1.0])
    return pack(d).astype(np.float32)
