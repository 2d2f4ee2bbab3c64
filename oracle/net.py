"""FP64 oracle of the CoNet receiver network, its BCE loss, backward pass and Adam.

Architecture (Sec. III, Fig. "Example I", Fig. RB, Fig. MRB; readings O7-O13):

* Branch 0 is the main net, branches 1..M the support nets; every branch sees the
  whole input grid (Sec. III: the TTI is processed concurrently by all subnets), unless
  ``support_inputs`` = 1: then the support nets are fed only the pilot information (Sec.
  III's generalisation: subsets of the inputs, such as the pilot symbols, fed selectively
  to supporting nets).  Their input layers read the pilot mask and the LS estimate at the
  pilots but not the received signal: the weights on the Re / Im Y channels of every
  antenna are held at zero (reading O15); ``support_mask`` names another subset of the
  input channels (bit j = channel j fed).
* Input layer of every branch: 3x3 conv + bias + ReLU.
* Plain networks: ``depth`` 3x3 conv + ReLU layers per branch (the input layer
  included).  Residual networks: input layer then ``depth`` blocks; support branches
  use the pre-activation residual block RB (LN -> ReLU -> conv -> LN -> ReLU -> conv,
  plus the skip), the main branch the modified block MRB (the RB without its first
  normalisation, because its input was normalised right after the fusion).
* Fusion after layer / block i (bit i of ``fuse_mask``): the main activation becomes
  the element-wise (Hadamard) product of the main and all support activations (or,
  ``fuse_op``, their sum or, in plain networks, their concatenation over channels, reading
  R9, which the main's next layer then reads with n_branches x width input channels),
  followed by LayerNorm over channels when ``norm`` is set; the support branches
  continue with their own unfused activations.
* Head: 1x1 conv of the main activation to Q LLRs per resource element.

3x3 convolutions are 'same' (zero padding 1 on the symbol and subcarrier axes), with
bias, weights laid out [C_out][3][3][C_in] and activations channels-last [B,T,F,C].
A tiny reverse-mode tape gives the gradients; every op's backward is its textbook
derivative.  LayerNorm uses eps = 1e-5.
"""
from __future__ import annotations

import numpy as np

LN_EPS = 1e-5
ADAM_BETA1 = 0.9
ADAM_BETA2 = 0.999
ADAM_EPS = 1e-8


# ----------------------------------------------------------------------------- parameters
def fused_width(cfg, i):
    """Channels of the main activation after fusion point i: n_branches x width where the
    point concatenates (fuse_op 2), else width."""
    return cfg.n_branches * cfg.width if getattr(cfg, "fuse_op", 0) == 2 and cfg.fused(i) else cfg.width


def param_layout(cfg):
    """Ordered list of (name, shape) of the flat float parameter vector."""
    C, Q = cfg.width, cfg.qam_bits
    out = []
    for b in range(cfg.n_branches):
        out += [(f"b{b}.in.w", (C, 3, 3, cfg.c_in)), (f"b{b}.in.b", (C,))]
        if not cfg.residual:
            for l in range(1, cfg.depth):
                cin = fused_width(cfg, l - 1) if b == 0 else C
                out += [(f"b{b}.l{l}.w", (C, 3, 3, cin)), (f"b{b}.l{l}.b", (C,))]
        else:
            for k in range(cfg.depth):
                if b >= 1 or cfg.resnet_baseline:
                    out += [(f"b{b}.k{k}.ln1.g", (C,)), (f"b{b}.k{k}.ln1.b", (C,))]
                if getattr(cfg, "depthwise", 0):
                    # depthwise-separable convs: a per-channel 3x3 then a 1x1 with bias
                    out += [(f"b{b}.k{k}.c1.dw", (C, 3, 3)), (f"b{b}.k{k}.c1.w", (C, C)), (f"b{b}.k{k}.c1.b", (C,)),
                            (f"b{b}.k{k}.ln2.g", (C,)), (f"b{b}.k{k}.ln2.b", (C,)),
                            (f"b{b}.k{k}.c2.dw", (C, 3, 3)), (f"b{b}.k{k}.c2.w", (C, C)), (f"b{b}.k{k}.c2.b", (C,))]
                else:
                    out += [(f"b{b}.k{k}.c1.w", (C, 3, 3, C)), (f"b{b}.k{k}.c1.b", (C,)),
                            (f"b{b}.k{k}.ln2.g", (C,)), (f"b{b}.k{k}.ln2.b", (C,)),
                            (f"b{b}.k{k}.c2.w", (C, 3, 3, C)), (f"b{b}.k{k}.c2.b", (C,))]
    if cfg.norm:
        n_points = cfg.depth + 1 if cfg.residual else cfg.depth
        for i in range(n_points):
            if cfg.fused(i):
                out += [(f"f{i}.g", (fused_width(cfg, i),)), (f"f{i}.b", (fused_width(cfg, i),))]
    head_c = C if cfg.residual else fused_width(cfg, cfg.depth - 1)
    out += [("head.w", (Q, head_c)), ("head.b", (Q,))]
    return out


def param_count(cfg) -> int:
    return int(sum(np.prod(s) for _, s in param_layout(cfg)))


def unflatten(cfg, flat):
    P, o = {}, 0
    for name, shape in param_layout(cfg):
        n = int(np.prod(shape))
        P[name] = flat[o:o + n].reshape(shape)
        o += n
    assert o == flat.size, (o, flat.size)
    return P


def init_params(cfg, seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in), fan_in = 9 C_in for 3x3 convs, C for the
    head), zero biases, LayerNorm gain 1 and shift 0 (O13 reading)."""
    g = np.random.default_rng(seed)
    parts = []
    for name, shape in param_layout(cfg):
        if name.endswith(".dw"):
            parts.append(g.standard_normal(shape).ravel() * np.sqrt(2.0 / 9.0))
        elif name.endswith(".w"):
            fan_in = int(np.prod(shape[1:]))
            parts.append(g.standard_normal(shape).ravel() * np.sqrt(2.0 / fan_in))
        elif name.endswith(".g"):
            parts.append(np.ones(int(np.prod(shape))))
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(parts)


# ----------------------------------------------------------------------------- tape
class Tape:
    """Minimal reverse-mode recorder: values, and per op (inputs, backward fn)."""

    def __init__(self):
        self.vals, self.recs = [], []

    def leaf(self, v):
        self.vals.append(v)
        self.recs.append(None)
        return len(self.vals) - 1

    def op(self, v, inputs, grad_fn):
        self.vals.append(v)
        self.recs.append((inputs, grad_fn))
        return len(self.vals) - 1

    def __getitem__(self, i):
        return self.vals[i]

    def backward(self, out, g_out):
        grads = {out: g_out}
        for i in range(len(self.vals) - 1, -1, -1):
            rec = self.recs[i]
            if rec is None or i not in grads:
                continue
            inputs, fn = rec
            for j, g in zip(inputs, fn(grads[i])):
                grads[j] = grads[j] + g if j in grads else g
        return grads


def _pad(x):
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))


def conv3x3(tp, x, w, b):
    X, W, bias = tp[x], tp[w], tp[b]
    B, T, F, _ = X.shape
    Xp = _pad(X)
    out = np.broadcast_to(bias, (B, T, F, W.shape[0])).copy()
    for kh in range(3):
        for kw in range(3):
            out += Xp[:, kh:kh + T, kw:kw + F, :] @ W[:, kh, kw, :].T

    def grad(g):
        dXp = np.zeros_like(Xp)
        dW = np.zeros_like(W)
        for kh in range(3):
            for kw in range(3):
                dXp[:, kh:kh + T, kw:kw + F, :] += g @ W[:, kh, kw, :]
                dW[:, kh, kw, :] = np.einsum("btfo,btfi->oi", g, Xp[:, kh:kh + T, kw:kw + F, :])
        return dXp[:, 1:T + 1, 1:F + 1, :], dW, g.sum(axis=(0, 1, 2))

    return tp.op(out, (x, w, b), grad)


def conv3x3_rounded(tp, x, w, b, q, data_grad=True):
    """The 3x3 conv of a 16-bit training step (the BF16 training recipe of the training
    workload: all conv math on BF16 operands, FP32 everything else): the output uses the
    rounded input and weight, q.act(x) and q.weight(w); the data gradient is the transposed
    conv of the rounded upstream gradient q.grad(g) with the rounded weight; the weight
    gradient correlates the rounded upstream gradient with the rounded input.  With identity
    roundings this is conv3x3 exactly."""
    X, W, bias = tp[x], tp[w], tp[b]
    Xq, Wq = q.act(X), q.weight(W)
    B, T, F, _ = X.shape
    Xp, Xqp = _pad(X), _pad(Xq)
    out = np.broadcast_to(bias, (B, T, F, W.shape[0])).copy()
    for kh in range(3):
        for kw in range(3):
            out += Xqp[:, kh:kh + T, kw:kw + F, :] @ Wq[:, kh, kw, :].T

    def grad(g):
        gq = q.grad(g)
        dXp = np.zeros_like(Xp)
        dW = np.zeros_like(W)
        for kh in range(3):
            for kw in range(3):
                if data_grad:
                    dXp[:, kh:kh + T, kw:kw + F, :] += gq @ Wq[:, kh, kw, :]
                dW[:, kh, kw, :] = np.einsum("btfo,btfi->oi", gq, Xqp[:, kh:kh + T, kw:kw + F, :])
        return dXp[:, 1:T + 1, 1:F + 1, :], dW, g.sum(axis=(0, 1, 2))

    return tp.op(out, (x, w, b), grad)


def dwconv3x3(tp, x, w):
    """Depthwise 3x3 'same' conv: out[..., c] = sum over (kh, kw) of x shifted by (kh - 1,
    kw - 1) (zero outside) times w[c, kh, kw]; no bias (the following 1x1 conv has one)."""
    X, W = tp[x], tp[w]
    B, T, F, _ = X.shape
    Xp = _pad(X)
    out = np.zeros_like(X)
    for kh in range(3):
        for kw in range(3):
            out += Xp[:, kh:kh + T, kw:kw + F, :] * W[:, kh, kw]

    def grad(g):
        dXp = np.zeros_like(Xp)
        dW = np.zeros_like(W)
        for kh in range(3):
            for kw in range(3):
                dXp[:, kh:kh + T, kw:kw + F, :] += g * W[:, kh, kw]
                dW[:, kh, kw] = np.einsum("btfc,btfc->c", g, Xp[:, kh:kh + T, kw:kw + F, :])
        return dXp[:, 1:T + 1, 1:F + 1, :], dW

    return tp.op(out, (x, w), grad)


def relu(tp, x):
    X = tp[x]

    def grad(g):
        return (g * (X > 0),)

    return tp.op(np.maximum(X, 0.0), (x,), grad)


def layernorm(tp, x, gam, bet):
    X, G, Bt = tp[x], tp[gam], tp[bet]
    mu = X.mean(-1, keepdims=True)
    var = ((X - mu) ** 2).mean(-1, keepdims=True)
    r = 1.0 / np.sqrt(var + LN_EPS)
    xh = (X - mu) * r

    def grad(g):
        dxh = g * G
        dx = r * (dxh - dxh.mean(-1, keepdims=True) - xh * (dxh * xh).mean(-1, keepdims=True))
        return dx, (g * xh).sum(axis=(0, 1, 2)), g.sum(axis=(0, 1, 2))

    return tp.op(xh * G + Bt, (x, gam, bet), grad)


def hadamard(tp, xs):
    vals = [tp[x] for x in xs]
    out = vals[0].copy()
    for v in vals[1:]:
        out = out * v

    def grad(g):
        gs = []
        for j in range(len(vals)):
            o = g.copy()
            for i, v in enumerate(vals):
                if i != j:
                    o = o * v
            gs.append(o)
        return tuple(gs)

    return tp.op(out, tuple(xs), grad)


def add(tp, x, y):
    return tp.op(tp[x] + tp[y], (x, y), lambda g: (g, g))


def concat(tp, xs):
    """Concatenation over the channel axis, branch 0 first."""
    vals = [tp[x] for x in xs]
    sizes = np.cumsum([v.shape[-1] for v in vals])[:-1]
    return tp.op(np.concatenate(vals, axis=-1), tuple(xs), lambda g: tuple(np.split(g, sizes, axis=-1)))


def add_all(tp, xs):
    out = xs[0]
    for x in xs[1:]:
        out = add(tp, out, x)
    return out


def head1x1(tp, x, w, b):
    X, W, bias = tp[x], tp[w], tp[b]

    def grad(g):
        return g @ W, np.einsum("btfq,btfc->qc", g, X), g.sum(axis=(0, 1, 2))

    return tp.op(X @ W.T + bias, (x, w, b), grad)


# ----------------------------------------------------------------------------- network
def forward(cfg, flat, X0, keep_tape=False, quant=None, taps=None):
    """LLR [B, T, F, Q] of the CoNet described by ``cfg`` with flat parameters ``flat``.

    ``quant`` (optional): an object whose ``act(x)`` and ``weight(w)`` replace every 3x3
    conv's input and weight by their quantised values (oracle.fp8, oracle.half).  When it
    also has ``grad(g)`` (oracle.half.Round16Train), the convs stay differentiable as in
    conv3x3_rounded; otherwise the quantised operands are tape leaves (inference only).
    ``taps`` (optional dict): receives, per fusion point i followed by a LayerNorm, the
    variance over channels of the fused product at every RE, taps[i] = [B, T, F]."""
    if getattr(cfg, "fuse_op", 0) == 2 and cfg.residual:
        raise ValueError("concatenation fuses plain networks only (a residual stream keeps its width)")
    tp = Tape()
    P = unflatten(cfg, np.asarray(flat, dtype=np.float64))
    ids = {k: tp.leaf(v) for k, v in P.items()}
    x_in = tp.leaf(np.asarray(X0, dtype=np.float64))
    nb = cfg.n_branches

    def conv(x, w, b):
        if quant is not None and hasattr(quant, "grad"):
            return conv3x3_rounded(tp, x, w, b, quant, data_grad=x != x_in)
        if quant is not None:
            x = tp.leaf(quant.act(tp[x]))
            w = tp.leaf(quant.weight(tp[w]))
        return conv3x3(tp, x, w, b)

    def fuse(i, acts):
        # fusion point i: the main activation becomes the interaction of all branches' (the
        # product, or the sum, reading the interaction operations of Sec. III), normalised;
        # supports keep their own activation, plus the main's with Example II's feedback
        if not cfg.fused(i):
            return list(acts)
        op = getattr(cfg, "fuse_op", 0)
        m = add_all(tp, acts) if op == 1 else concat(tp, acts) if op == 2 else hadamard(tp, acts)
        if cfg.norm:
            if taps is not None:
                taps[i] = tp[m].var(axis=-1)
            m = layernorm(tp, m, ids[f"f{i}.g"], ids[f"f{i}.b"])
        if getattr(cfg, "feedback", 0):
            return [m] + [add(tp, a, acts[0]) for a in acts[1:]]
        return [m] + list(acts[1:])

    def block_conv(x, name):
        # a residual block's conv: standard 3x3, or depthwise-separable (per-channel 3x3, then
        # 1x1 with bias: "depthwise convolutions" of Sec. II-A / III)
        if getattr(cfg, "depthwise", 0):
            if quant is not None and not hasattr(quant, "grad"):
                # reduced-precision operands (reading R8): the per-channel 3x3 reads the
                # activation in the operand format with its weights in full precision, its
                # output is stored in the operand format, and the 1x1 takes operand-format
                # weights
                xq = tp.leaf(quant.act(tp[x]))
                d = tp.leaf(quant.act(tp[dwconv3x3(tp, xq, ids[name + ".dw"])]))
                wq = tp.leaf(quant.weight(tp[ids[name + ".w"]]))
                return head1x1(tp, d, wq, ids[name + ".b"])
            return head1x1(tp, dwconv3x3(tp, x, ids[name + ".dw"]), ids[name + ".w"], ids[name + ".b"])
        return conv(x, ids[name + ".w"], ids[name + ".b"])

    def input_w(b):
        # selective support inputs: the support net's weights on the received-signal
        # channels (the first 2 n_rx) are zero, and so is their gradient
        w = ids[f"b{b}.in.w"]
        if b == 0 or not getattr(cfg, "support_inputs", 0):
            return w
        # the channels fed: support_mask's bits, by default the pilot information (pilot
        # mask and LS estimate, channels 2 N .. 2 N + 2)
        keep = getattr(cfg, "support_mask", 0) or (7 << (2 * cfg.n_rx))
        M = np.ones(P[f"b{b}.in.w"].shape)
        for j in range(cfg.c_in):
            if not (keep >> j) & 1:
                M[..., j] = 0.0
        return tp.op(tp[w] * M, (w,), lambda g: (g * M,))

    acts = [relu(tp, conv(x_in, input_w(b), ids[f"b{b}.in.b"])) for b in range(nb)]
    x = fuse(0, acts)
    if not cfg.residual:
        for l in range(1, cfg.depth):
            acts = [relu(tp, conv(x[b], ids[f"b{b}.l{l}.w"], ids[f"b{b}.l{l}.b"]))
                    for b in range(nb)]
            x = fuse(l, acts)
    else:
        for k in range(cfg.depth):
            u = []
            for b in range(nb):
                p = f"b{b}.k{k}."
                if b >= 1 or cfg.resnet_baseline:
                    h1 = relu(tp, layernorm(tp, x[b], ids[p + "ln1.g"], ids[p + "ln1.b"]))
                else:
                    h1 = relu(tp, x[b])
                t1 = block_conv(h1, p + "c1")
                h2 = relu(tp, layernorm(tp, t1, ids[p + "ln2.g"], ids[p + "ln2.b"]))
                u.append(add(tp, x[b], block_conv(h2, p + "c2")))
            x = fuse(k + 1, u)
    llr = head1x1(tp, x[0], ids["head.w"], ids["head.b"])
    if keep_tape:
        return tp[llr], (tp, llr, ids, x_in)
    return tp[llr]


def bce_loss(llr, bits, pilot_mask):
    """Mean BCE-with-logits over data REs and bits, and its gradient w.r.t. the LLRs:
    l = softplus(L) - b L = max(L, 0) - b L + log1p(exp(-|L|)); dl/dL = sigmoid(L) - b."""
    data = (~pilot_mask.astype(bool))[None, :, :, None]
    count = llr.shape[0] * int(data.sum()) * llr.shape[-1]
    b = bits.astype(np.float64)
    per = np.maximum(llr, 0.0) - b * llr + np.log1p(np.exp(-np.abs(llr)))
    loss = float((per * data).sum() / count)
    sig = 1.0 / (1.0 + np.exp(-llr))
    dllr = (sig - b) * data / count
    return loss, dllr


def backward(cfg, tape_info, dllr):
    """Flat parameter gradient (same layout as the parameters) and dX0 for dLLR."""
    tp, out, ids, x_in = tape_info
    grads = tp.backward(out, np.asarray(dllr, dtype=np.float64))
    parts = []
    for name, shape in param_layout(cfg):
        g = grads.get(ids[name])
        parts.append(np.zeros(int(np.prod(shape))) if g is None else np.asarray(g).ravel())
    return np.concatenate(parts), grads.get(x_in)


def loss_and_grad(cfg, flat, X0, bits, pilot_mask):
    llr, info = forward(cfg, flat, X0, keep_tape=True)
    loss, dllr = bce_loss(llr, bits, pilot_mask)
    g, _ = backward(cfg, info, dllr)
    return loss, g, llr


def adam_step(w, g, m, v, step: int, lr: float, beta1=ADAM_BETA1, beta2=ADAM_BETA2, eps=ADAM_EPS):
    """One bias-corrected Adam update (Kingma & Ba 2015), ``step`` counted from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
