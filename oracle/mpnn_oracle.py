"""FP64 NumPy restatement of the learned restart proposal network — TEST
INFRASTRUCTURE ONLY (used by tests/ to check the CUDA forward and backward).

The architecture, features and parameter layout are the ones documented at
ffsat_mpnn_create in include/ffsat.h; this file shares no code with the CUDA
library.  Weights can be rounded to BF16 (round to nearest even) to mirror the
kernels' weight precision, and the inputs of every dense product (activations
in the forward pass, back-propagated gradients and activations in the
backward pass) likewise, as the tensor-core dense layers take BF16 operands
with FP32 sums; biases, bias gradients, aggregations and the output head stay
unrounded."""
from __future__ import annotations

import numpy as np

H = 64
FV = FC = 8


def layout(layers: int):
    off = 0
    out = {}

    def take(name, shape):
        nonlocal off
        size = int(np.prod(shape))
        out[name] = (off, shape)
        off += size

    take("Wv0", (H, FV))
    take("bv0", (H,))
    take("Wc0", (H, FC))
    take("bc0", (H,))
    for l in range(layers):
        take(f"A{l}", (H, H))
        take(f"Uc{l}", (H, 2 * H))
        take(f"buc{l}", (H,))
        take(f"B{l}", (H, H))
        take(f"Uv{l}", (H, 2 * H))
        take(f"buv{l}", (H,))
    take("wo", (H,))
    take("bo", (1,))
    return out, off


def unpack(p, layers):
    lay, _ = layout(layers)
    return {k: np.asarray(p[o:o + int(np.prod(s))], dtype=np.float64).reshape(s) for k, (o, s) in lay.items()}


def bf16(x):
    """Round float values to the nearest BF16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def graph(inst):
    """Incidence with signs, features and normalisers from the documented definitions."""
    n, m = inst.n, inst.m
    rows, cols, sgn = [], [], []
    pos = np.zeros(n); neg = np.zeros(n); nx = np.zeros(n); cpos = np.zeros(n); cneg = np.zeros(n)
    fc = np.zeros((m, FC))
    for c in range(m):
        t, p, ls = inst.constraint(c)
        L = len(ls)
        for l in ls:
            v = abs(int(l)) - 1
            rows.append(c); cols.append(v); sgn.append(1.0 if l > 0 else -1.0)
            if t == 0:
                (pos if l > 0 else neg)[v] += 1
            elif t == 1:
                nx[v] += 1
            else:
                (cpos if l > 0 else cneg)[v] += 1
        fc[c] = [1, t == 0, t == 1, t == 2, L / 10.0, (1.0 if p & 1 else -1.0) if t == 1 else 0.0,
                 p / L if t == 2 else 0.0, 0]
    rows = np.array(rows); cols = np.array(cols); sgn = np.array(sgn)
    S = np.zeros((m, n))
    np.add.at(S, (rows, cols), sgn)
    deg = np.abs(S).sum(axis=0)
    ln = np.abs(S).sum(axis=1)
    mean_deg = inst.nnz / n
    fv = np.zeros((n, FV))
    fv[:, 0] = 1
    fv[:, 1] = pos / mean_deg
    fv[:, 2] = neg / mean_deg
    fv[:, 3] = (pos - neg) / (pos + neg + 1)
    fv[:, 4] = nx / mean_deg
    fv[:, 5] = (cpos - cneg) / (cpos + cneg + 1)
    fv[:, 6] = deg / mean_deg
    return S, fv, fc, deg, ln


def _identity(a):
    return a


def forward(P, G, layers, q=_identity):
    """q rounds the inputs of each dense product (bf16, or the identity)."""
    S, fv, fc, deg, ln = G
    Sc = S / ln[:, None]                                   # mean over a constraint's literals
    Sv = (S / np.where(deg > 0, deg, 1)[None, :]).T        # mean over a variable's occurrences
    cache = {}
    relu = lambda a: np.maximum(a, 0.0)
    hv = relu(q(fv) @ P["Wv0"].T + P["bv0"]); hc = relu(q(fc) @ P["Wc0"].T + P["bc0"])
    cache["hv0"], cache["hc0"] = hv, hc
    for l in range(layers):
        mc = Sc @ (q(hv) @ P[f"A{l}"].T)
        hc_new = relu(q(np.concatenate([hc, mc], 1)) @ P[f"Uc{l}"].T + P[f"buc{l}"])
        mv = Sv @ (q(hc_new) @ P[f"B{l}"].T)
        hv_new = relu(q(np.concatenate([hv, mv], 1)) @ P[f"Uv{l}"].T + P[f"buv{l}"])
        cache[f"mc{l}"], cache[f"mv{l}"] = mc, mv
        cache[f"hc{l + 1}"], cache[f"hv{l + 1}"] = hc_new, hv_new
        hv, hc = hv_new, hc_new
    z = hv @ P["wo"] + P["bo"][0]
    return z, cache


def loss_and_grad(p, inst, target, layers, bf16_weights=True, bf16_inputs=True):
    """Loss mean softplus(-t z) and its gradient w.r.t. the parameter vector
    (w.r.t. the BF16-rounded weights when bf16_weights, and with the inputs of
    every dense product rounded to BF16 when bf16_inputs, as the kernels
    compute)."""
    q = bf16 if bf16_inputs else _identity
    P = unpack(p, layers)
    if bf16_weights:
        for k in P:
            if not k.startswith("b"):
                P[k] = bf16(P[k])
    G = graph(inst)
    S, fv, fc, deg, ln = G
    Sc = S / ln[:, None]
    Sv = (S / np.where(deg > 0, deg, 1)[None, :]).T
    z, cache = forward(P, G, layers, q)
    t = np.asarray(target, dtype=np.float64)
    n = len(z)
    u = -t * z
    loss = np.mean(np.logaddexp(0.0, u))
    dz = -t / (1.0 + np.exp(-u)) / n
    g = {k: np.zeros_like(v) for k, v in P.items()}
    hv = cache[f"hv{layers}"]
    g["wo"] = dz @ hv
    g["bo"] = np.array([dz.sum()])
    dhv = np.outer(dz, P["wo"])
    dhc = np.zeros_like(cache[f"hc{layers}"])
    for l in reversed(range(layers)):
        hv_prev, hc_prev = cache[f"hv{l}"], cache[f"hc{l}"]
        hv_l, hc_l = cache[f"hv{l + 1}"], cache[f"hc{l + 1}"]
        mv, mc = cache[f"mv{l}"], cache[f"mc{l}"]
        d = dhv * (hv_l > 0)
        g[f"Uv{l}"] += q(d).T @ q(np.concatenate([hv_prev, mv], 1))
        g[f"buv{l}"] += d.sum(0)
        dcat = q(d) @ P[f"Uv{l}"]
        dhv_prev, dmv = dcat[:, :H], dcat[:, H:]
        dtc = Sv.T @ dmv
        g[f"B{l}"] += q(dtc).T @ q(hc_l)
        dhc = dhc + q(dtc) @ P[f"B{l}"]
        d = dhc * (hc_l > 0)
        g[f"Uc{l}"] += q(d).T @ q(np.concatenate([hc_prev, mc], 1))
        g[f"buc{l}"] += d.sum(0)
        dcat = q(d) @ P[f"Uc{l}"]
        dhc_prev, dmc = dcat[:, :H], dcat[:, H:]
        dtv = Sc.T @ dmc
        g[f"A{l}"] += q(dtv).T @ q(hv_prev)
        dhv = dhv_prev + q(dtv) @ P[f"A{l}"]
        dhc = dhc_prev
    d = dhv * (cache["hv0"] > 0)
    g["Wv0"] += q(d).T @ q(fv)
    g["bv0"] += d.sum(0)
    d = dhc * (cache["hc0"] > 0)
    g["Wc0"] += q(d).T @ q(fc)
    g["bc0"] += d.sum(0)
    lay, total = layout(layers)
    flat = np.zeros(total)
    for k, (o, s) in lay.items():
        flat[o:o + int(np.prod(s))] = g[k].reshape(-1)
    return loss, flat, np.tanh(z)
