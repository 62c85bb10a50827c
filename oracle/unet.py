"""Float64 reference of the learned pressure correction network.

Oracle (test infrastructure only).  The paper has no learned component; the
network is the 3-D U-Net described for the learned pressure-multigrid
correction: three levels (widths c0, c1, c2 = 16/32/64), two 3x3x3
convolutions with ReLU per level, 2x2x2 average pooling down, nearest
up-sampling with skip concatenation up, and a 1x1x1 head to one channel.

Tensors are [C, Z, Y, X] float64; convolutions use zero padding 1.
Weights: W[o, c, dz, dy, dx], bias b[o].  forward() returns the output and a
tape; backward() returns the gradients of 0.5 * mean((out - target)^2).

Both take an optional storage rounding `rnd` applied wherever a tensor is
stored between operations (convolution and pooling outputs, the gradients
passed between layers), so that a network whose kernels store activations in
bfloat16 can be compared with the same storage decisions (`bf16` below).
Arithmetic stays float64; the default is no rounding.
"""
import numpy as np


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), via float32: the value a
    float32 accumulator would hold, then its upper 16 bits with
    round-to-nearest-even on the lower 16."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def _ident(a):
    return a

LAYERS = ("a1", "a2", "b1", "b2", "c1", "c2", "ub1", "ub2", "ua1", "ua2")


def layer_shapes(cin=3, c0=16, c1=32, c2=64):
    """(C_out, C_in) of every 3x3x3 convolution, then the head."""
    return {"a1": (c0, cin), "a2": (c0, c0), "b1": (c1, c0), "b2": (c1, c1), "c1": (c2, c1), "c2": (c2, c2),
            "ub1": (c1, c2 + c1), "ub2": (c1, c1), "ua1": (c0, c1 + c0), "ua2": (c0, c0), "head": (1, c0)}


def init_params(rng, cin=3, c0=16, c1=32, c2=64):
    p = {}
    for name, (co, ci) in layer_shapes(cin, c0, c1, c2).items():
        k = 1 if name == "head" else 3
        fan = ci * k ** 3
        p[name + ".w"] = rng.standard_normal((co, ci, k, k, k)) * np.sqrt(2.0 / fan)
        p[name + ".b"] = np.zeros(co)
    return p


def conv3(x, w, b):
    """3x3x3 convolution, zero padding 1: out[o] = b[o] + sum_c,taps w * x."""
    co = w.shape[0]
    Z, Y, X = x.shape[1:]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.broadcast_to(b[:, None, None, None], (co, Z, Y, X)).copy()
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                win = xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X]
                out += np.tensordot(w[:, :, dz, dy, dx], win, axes=([1], [0]))
    return out


def conv3_backward(x, w, dout):
    """Gradients of conv3 with respect to x, w and b."""
    Z, Y, X = x.shape[1:]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                win = xp[:, dz:dz + Z, dy:dy + Y, dx:dx + X]
                dw[:, :, dz, dy, dx] = np.tensordot(dout, win, axes=([1, 2, 3], [1, 2, 3]))
                dxp[:, dz:dz + Z, dy:dy + Y, dx:dx + X] += np.tensordot(w[:, :, dz, dy, dx], dout, axes=([0], [0]))
    return dxp[:, 1:-1, 1:-1, 1:-1], dw, dout.sum(axis=(1, 2, 3))


def pool(x):
    C, Z, Y, X = x.shape
    return x.reshape(C, Z // 2, 2, Y // 2, 2, X // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(d, shape):
    return np.repeat(np.repeat(np.repeat(d, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up_backward(d):
    C, Z, Y, X = d.shape
    return d.reshape(C, Z // 2, 2, Y // 2, 2, X // 2, 2).sum(axis=(2, 4, 6))


def forward(p, x, rnd=None):
    R = rnd or _ident
    t = {"x": x}

    def cr(name, inp):
        pre = conv3(inp, p[name + ".w"], p[name + ".b"])
        out = R(np.maximum(pre, 0.0))
        t[name + ".in"] = inp
        t[name + ".out"] = out
        return out

    a = cr("a2", cr("a1", x))
    b = cr("b2", cr("b1", R(pool(a))))
    c = cr("c2", cr("c1", R(pool(b))))
    ub = cr("ub2", cr("ub1", np.concatenate([up(c), b], axis=0)))
    ua = cr("ua2", cr("ua1", np.concatenate([up(ub), a], axis=0)))
    w = p["head.w"][:, :, 0, 0, 0]
    out = np.tensordot(w, ua, axes=([1], [0])) + p["head.b"][:, None, None, None]
    t["head.in"] = ua
    t["a"], t["b"], t["c"], t["ub"] = a, b, c, ub
    return out, t


def loss(out, target):
    return 0.5 * np.mean((out - target) ** 2)


def backward(p, t, out, target, rnd=None):
    R = rnd or _ident
    g = {}
    dout = (out - target) / out.size
    ua = t["head.in"]
    w = p["head.w"][:, :, 0, 0, 0]
    g["head.w"] = np.tensordot(dout, ua, axes=([1, 2, 3], [1, 2, 3]))[:, :, None, None, None]
    g["head.b"] = dout.sum(axis=(1, 2, 3))
    d = R(np.tensordot(w, dout, axes=([0], [0])))

    def crb(name, d):
        d = d * (t[name + ".out"] > 0.0)
        dx, dw, db = conv3_backward(t[name + ".in"], p[name + ".w"], d)
        g[name + ".w"], g[name + ".b"] = dw, db
        return R(dx)

    c1 = t["b"].shape[0]
    d = crb("ua1", crb("ua2", d))
    d_up_ub, d_a_skip = d[:c1], d[c1:]
    d = crb("ub1", crb("ub2", R(up_backward(d_up_ub))))
    d_up_c, d_b_skip = d[:t["c"].shape[0]], d[t["c"].shape[0]:]
    d = crb("c1", crb("c2", R(up_backward(d_up_c))))
    d = R(pool_backward(d, None) + d_b_skip)
    d = crb("b1", crb("b2", d))
    d = R(pool_backward(d, None) + d_a_skip)
    dx = crb("a1", crb("a2", d))
    return g, dx
