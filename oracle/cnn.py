"""CPU oracle of the learned Poisson warm start -- TEST INFRASTRUCTURE ONLY.

Only the tests may import this module.  Plain numpy in float64, written from
the definitions below; it shares nothing with the CUDA library.

The warm start is not part of the paper's method: it predicts the potential
of Eq. (8) from the charge density so that the multigrid solve starts close
to its answer.  Definitions used here (and by the library):

Training pair of one r-z run (node arrays of shape (nz + 1, nr + 1)),
z_i = i dz, L = nz dz (the gap), absolute form:
    d = rho,  base = V z / L     (the charge-free solution of Eq. (8): linear in z)
delta form, against the previous solve (rho', phi', V'):
    d = rho - rho',  base = phi' + (V - V') z / L
and for both, with m = max |d|:
    x = d / m                                          (0 where m = 0)
    t = (phi - base) eps0 / (m dz^2)
and the warm start built from a prediction y of t:
    phi_0 = base + y m dz^2 / eps0.
Dividing by dz^2 gives the potential in grid units of the unit-spacing
Laplacian, the scale a convolution over the grid sees.

Network: six 3 x 3 convolutions over the node grid, output the size of the
input (zero padding), channels 1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU
after the first five, one bias per output channel:
    a_l[p, co] = b_l[co] + sum_{dy, dx, ci} W_l[tap(dy, dx), co, ci] h_{l-1}[p + (dy, dx), ci]
    h_l = relu(a_l) (l < 6),  y = a_6,  tap(dy, dx) = 3 (dy + 1) + (dx + 1)
with h_{l-1} = 0 outside the grid (cross-correlation, as in deep-learning
convolutions).  Parameter vector: for l = 1..6 in order, W_l as
[tap][co][ci] followed by b_l[co].

Loss: mean over the batch and the nodes of (y - t)^2.

Extrapolated form, against the two previous solves (rho', phi', V') and
(rho'', phi'', V''): the start is the potential extrapolated linearly in
time, and the network corrects it from the charge that the extrapolation
misses:
    d = rho - (2 rho' - rho''),
    base = 2 phi' - phi'' + (V - 2 V' + V'') z / L.
Its training loss is the residual of Eq. (8) that the corrected start
leaves, in the units of the finite-volume equations: on the interior rows
(the electrode rows are Dirichlet, y = 0 there)
    r = w x - S y,
    (S y)_ij = (a+_j + a-_j + 2 w_j) y_ij - a+_j y_i,j+1 - a-_j y_i,j-1
               - w_j (y_i+1,j + y_i-1,j),
with, for dz = dr (radial node j = 0..nr, outer radius R = nr dr), the
face coefficients and volumes of the finite-volume r-z Laplacian divided by
2 pi dr: a+_j = j + 1/2 (0 at j = nr: Neumann), a-_j = j - 1/2 (0 on the
axis), w_j = j, 1/8 on the axis, nr/2 - 1/8 at the outer radius (the node's
finite volume over 2 pi dr^3).  S is symmetric; t of the pair satisfies
S t = w x exactly when phi solves Eq. (8).  Loss: sum of r^2 over the
interior nodes of the batch divided by their number.

Adam (Kingma and Ba, ICLR 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2)
g^2, w -= lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps) at step k = 1, 2, ...

bf16 mirror: with `bf16=True` the values are rounded to bfloat16 (round to
nearest, ties to even) where the library stores bfloat16 -- the weights
every layer uses, the activations h_1..h_5 and the loss gradients with
respect to a_1..a_5 -- so that the two sides differ only by the order of
their float sums.
"""
import numpy as np

CH = 32
LAYERS = ((1, CH), (CH, CH), (CH, CH), (CH, CH), (CH, CH), (CH, 1))   # (c_in, c_out)
EPS0 = 8.8541878128e-12


def layer_sizes():
    """(weights, biases) counts of the six layers."""
    return [(9 * co * ci, co) for ci, co in LAYERS]


def n_params():
    return sum(w + b for w, b in layer_sizes())


def unpack(params):
    """Parameter vector -> list of (W [9, co, ci], b [co]) per layer."""
    params = np.asarray(params, dtype=np.float64)
    out, o = [], 0
    for ci, co in LAYERS:
        W = params[o:o + 9 * co * ci].reshape(9, co, ci)
        o += 9 * co * ci
        b = params[o:o + co]
        o += co
        out.append((W, b))
    assert o == params.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def init_params(seed):
    """He-normal weights, zero biases (a seeded starting point)."""
    rng = np.random.default_rng(seed)
    layers = []
    for ci, co in LAYERS:
        W = rng.standard_normal((9, co, ci)) * np.sqrt(2.0 / (9 * ci))
        layers.append((W, np.zeros(co)))
    return pack(layers)


def round_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def shift(h, dy, dx):
    """s[b, i, j, :] = h[b, i + dy, j + dx, :], zero outside the grid."""
    B, H, W, C = h.shape
    s = np.zeros_like(h)
    i0, i1 = max(0, -dy), min(H, H - dy)
    j0, j1 = max(0, -dx), min(W, W - dx)
    s[:, i0:i1, j0:j1, :] = h[:, i0 + dy:i1 + dy, j0 + dx:j1 + dx, :]
    return s


TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv(h, W, b):
    """a[p, co] = b[co] + sum_tap sum_ci W[tap, co, ci] h[p + tap, ci]."""
    a = np.zeros(h.shape[:3] + (W.shape[1],)) + b
    for tap, (dy, dx) in enumerate(TAPS):
        a += shift(h, dy, dx) @ W[tap].T
    return a


def forward(params, x, bf16=False):
    """x [B, H, W] -> (y [B, H, W], list of layer inputs h_0..h_5)."""
    layers = unpack(params)
    rnd = round_bf16 if bf16 else (lambda v: v)
    h = np.asarray(x, dtype=np.float64)[..., None]
    hs = [h]
    for l, (W, b) in enumerate(layers):
        a = conv(h, rnd(W), b)
        if l < 5:
            h = rnd(np.maximum(a, 0.0))
            hs.append(h)
        else:
            y = a[..., 0]
    return y, hs


def loss(params, x, t, bf16=False):
    y, _ = forward(params, x, bf16)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def loss_and_grad(params, x, t, bf16=False):
    """Mean squared error and its gradient by back-propagation, in the
    parameter-vector layout."""
    layers = unpack(params)
    rnd = round_bf16 if bf16 else (lambda v: v)
    y, hs = forward(params, x, bf16)
    t = np.asarray(t, dtype=np.float64)
    N = y.size
    L = float(np.mean((y - t) ** 2))
    g = (2.0 / N) * (y - t)[..., None]          # dL/da_6
    grads = [None] * 6
    for l in range(5, -1, -1):
        W, _ = layers[l]
        Wr = rnd(W)
        h = hs[l]                                # input of layer l
        gW = np.zeros_like(W)
        for tap, (dy, dx) in enumerate(TAPS):
            # dL/dW[tap, co, ci] = sum_p g[p, co] h[p + tap, ci]
            gW[tap] = np.einsum("bijc,bijd->cd", g, shift(h, dy, dx))
        gb = g.sum(axis=(0, 1, 2))
        grads[l] = (gW, gb)
        if l == 0:
            break
        # dL/dh[q, ci] = sum_tap sum_co W[tap, co, ci] g[q - tap, co]
        gh = np.zeros(h.shape)
        for tap, (dy, dx) in enumerate(TAPS):
            gh += shift(g, -dy, -dx) @ Wr[tap]
        g = rnd(gh * (h > 0.0))                  # through the ReLU of layer l - 1
    return L, pack(grads)


def rz_weights(W):
    """(a+, a-, w) of the unit finite-volume r-z operator for W = nr + 1 radial nodes."""
    nr = W - 1
    j = np.arange(W, dtype=np.float64)
    ap = j + 0.5
    ap[nr] = 0.0
    am = j - 0.5
    am[0] = 0.0
    w = j.copy()
    w[0] = 1.0 / 8.0
    w[nr] = nr / 2.0 - 1.0 / 8.0
    return ap, am, w


def rz_operator(y):
    """S y on the interior rows of y [..., H, W] (rows 0 and H - 1 read as 0
    and returned 0)."""
    y = np.array(y, dtype=np.float64)
    y[..., 0, :] = 0.0
    y[..., -1, :] = 0.0
    ap, am, w = rz_weights(y.shape[-1])
    out = (ap + am + 2.0 * w) * y
    out[..., :, :-1] -= ap[:-1] * y[..., :, 1:]
    out[..., :, 1:] -= am[1:] * y[..., :, :-1]
    out[..., 1:, :] -= w * y[..., :-1, :]
    out[..., :-1, :] -= w * y[..., 1:, :]
    out[..., 0, :] = 0.0
    out[..., -1, :] = 0.0
    return out


def rz_residual(x, y):
    """r = w x - S y on the interior rows (0 on the electrode rows)."""
    x = np.asarray(x, dtype=np.float64)
    _, _, w = rz_weights(x.shape[-1])
    r = w * x - rz_operator(y)
    r[..., 0, :] = 0.0
    r[..., -1, :] = 0.0
    return r


def backprop(params, hs, g, bf16=False):
    """Parameter gradient in the packed layout from dL/da_6 = g [B, H, W, 1]
    and the layer inputs hs of forward()."""
    layers = unpack(params)
    rnd = round_bf16 if bf16 else (lambda v: v)
    grads = [None] * 6
    for l in range(5, -1, -1):
        W, _ = layers[l]
        Wr = rnd(W)
        h = hs[l]
        gW = np.zeros_like(W)
        for tap, (dy, dx) in enumerate(TAPS):
            gW[tap] = np.einsum("bijc,bijd->cd", g, shift(h, dy, dx))
        gb = g.sum(axis=(0, 1, 2))
        grads[l] = (gW, gb)
        if l == 0:
            break
        gh = np.zeros(h.shape)
        for tap, (dy, dx) in enumerate(TAPS):
            gh += shift(g, -dy, -dx) @ Wr[tap]
        g = rnd(gh * (h > 0.0))
    return pack(grads)


def resid_loss_and_grad(params, x, bf16=False):
    """Residual loss of the extrapolated form and its gradient: L = sum of
    r^2 over the interior nodes / their number; dL/dy = -(2 / N) S r."""
    y, hs = forward(params, x, bf16)
    r = rz_residual(x, y)
    n_int = y.shape[0] * (y.shape[1] - 2) * y.shape[2]
    L = float((r * r).sum() / n_int)
    g = (-2.0 / n_int) * rz_operator(r)
    return L, backprop(params, hs, g[..., None], bf16)


def training_pair_extrap(rho, phi, V, dz, rho1, phi1, V1, rho2, phi2, V2):
    """(x, t) of the extrapolated form from the solve (rho, phi, V) and the
    two before it (1: the previous one, 2: the one before)."""
    rho = np.asarray(rho, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    nz = rho.shape[0] - 1
    zL = (np.arange(nz + 1)[:, None] / nz) * np.ones_like(rho)
    d = rho - (2.0 * np.asarray(rho1, dtype=np.float64) - np.asarray(rho2, dtype=np.float64))
    base = 2.0 * np.asarray(phi1, dtype=np.float64) - np.asarray(phi2, dtype=np.float64) + \
        (V - 2.0 * V1 + V2) * zL
    m = np.abs(d).max()
    if m == 0.0:
        return np.zeros_like(rho), np.zeros_like(rho)
    return d / m, (phi - base) * EPS0 / (m * dz * dz)


def adam_step(params, grad, m, v, k, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step k (1-based); returns new (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** k)
    vh = v / (1.0 - b2 ** k)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def node_density(rho_int, weight, dz, dr, nz, nr):
    """Node charge density (C/m^3) of an r-z run from its fixed-point node
    charge (units of e 2^-32 per super-particle, electrons plus heavies):
    Verboncoeur's node volumes -- axis pi dz dr^2 / 3, interior 2 pi dz dr^2 j,
    outer wall 2 pi dz dr^2 (nr / 2 - 1 / 6) -- halved on the electrode rows."""
    j = np.arange(nr + 1, dtype=np.float64)
    vol = 2.0 * np.pi * dz * dr * dr * j
    vol[0] = np.pi * dz * dr * dr / 3.0
    vol[nr] = 2.0 * np.pi * dz * dr * dr * (nr / 2.0 - 1.0 / 6.0)
    vol = np.tile(vol, (nz + 1, 1))
    vol[0] *= 0.5
    vol[nz] *= 0.5
    q = np.asarray(rho_int, dtype=np.float64).reshape(nz + 1, nr + 1)
    return 1.602176634e-19 * weight * q / 2.0 ** 32 / vol


def training_pair(rho, phi, V, dz, rho_prev=None, phi_prev=None, V_prev=0.0):
    """(x, t) of one run from its node density rho (C/m^3) and potential phi
    (V), arrays of shape (nz + 1, nr + 1); the delta form when rho_prev and
    phi_prev (the previous solve's) are given."""
    rho = np.asarray(rho, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    nz = rho.shape[0] - 1
    zL = (np.arange(nz + 1)[:, None] / nz) * np.ones_like(rho)
    if rho_prev is None:
        d, base = rho, V * zL
    else:
        d = rho - np.asarray(rho_prev, dtype=np.float64)
        base = np.asarray(phi_prev, dtype=np.float64) + (V - V_prev) * zL
    m = np.abs(d).max()
    if m == 0.0:
        return np.zeros_like(rho), np.zeros_like(rho)
    return d / m, (phi - base) * EPS0 / (m * dz * dz)


def warm_start(y, m, V, dz, phi_prev=None, V_prev=0.0):
    """phi_0 (interior and electrode rows alike) from a prediction y of t."""
    y = np.asarray(y, dtype=np.float64)
    nz = y.shape[0] - 1
    zL = (np.arange(nz + 1)[:, None] / nz) * np.ones_like(y)
    base = V * zL if phi_prev is None else np.asarray(phi_prev, dtype=np.float64) + (V - V_prev) * zL
    return base + y * m * dz * dz / EPS0
