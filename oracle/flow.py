"""Plain FP64 numpy oracle of the learned proposal: an affine coupling flow
composed after the VEGAS map, and its training.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this module; the product path
(paper_2408_09229_gb300) never does.  It shares no code with the CUDA library.

The learned proposal is not part of cuVegas (arXiv 2408.09229).  The paper's
VEGAS+ map M (Sec. 2.1.1) samples x' = M(y); the flow F then maps x' to the
point x = F(x') where the integrand is evaluated, and the estimator uses
g(x') = f(F(x')) |det dF/dx'(x')|, whose integral over the unit cube equals
that of f, so the VEGAS+ machinery (Algorithms 1-2, Eqs. (2)-(9)) runs
unchanged on g.  The flow follows the affine coupling layers of RealNVP
(Dinh, Sohl-Dickstein, Bengio, "Density estimation using Real NVP", ICLR 2017)
between a logit and a sigmoid, so that it maps the open unit cube onto
itself; it is trained with Adam (Kingma and Ba, ICLR 2015).

Definitions (the same in the CUDA path):
  * L = 6 layers, hidden width H = 64.  Layer l conditions on the axes
    A_l = {k : k = l (mod 2)} and transforms B_l = the other axes.
  * Normalising direction N (x -> x'), the one the density is trained in:
      z = clamp(logit(x), -Z, Z), Z = 20
      for l = 0..L-1:  h = z[A_l];  a1 = W1 h + b1;  u1 = relu(a1);
                       a2 = W2 u1 + b2;  u2 = relu(a2);  o = W3 u2 + b3;
                       s_j = S tanh(o_{2j} / S) (S = 2),  t_j = o_{2j+1};
                       z[B_l] = z[B_l] exp(s) + t
      x' = sigmoid(z)
      log|det dN/dx| = sum_k ls(z_out,k) + sum_{l,j} s_{l,j} - sum_k ls(z_in,k),
      with ls(z) = log sigmoid'(z) = -|z| - 2 log(1 + exp(-|z|)).
  * Sampling direction F = N^-1 (x' -> x): the layers in reverse order with
    z[B_l] = (z[B_l] - t) exp(-s); log|det dF/dx'| = -(the same terms).
  * Training: samples x_i with weights w_i >= 0 (|g| of earlier VEGAS
    iterations, i.e. |f| over the proposal density); the loss is the weighted
    negative log-likelihood of the flow's density with a uniform base,
      loss = - sum_i w_i log|det dN/dx(x_i)| / sum_i w_i,
    whose minimiser makes the flow's density proportional to |f| (the
    forward KL divergence).
  * Parameters: one flat vector, per layer l in order
      W1 [H][a_l], b1 [H], W2 [H][H], b2 [H], W3 [2 b_l][H], b3 [2 b_l],
    row-major; rows 2j and 2j+1 of W3 give s_j and t_j.

bf16=True rounds what the CUDA path stores as bf16 (the weight matrices,
the conditioner input h and the hidden activations u1, u2; not the biases)
to bf16, round to nearest even, from their FP32 values; the arithmetic stays
FP64.  grad(..., bf16_grad=True) also rounds the backward operands that the
tensor-core gradient stores as bf16 (see grad).
"""
import numpy as np

LAYERS, HIDDEN, S_CLAMP, Z_CLAMP = 6, 64, 2.0, 20.0


def masks(d, layer):
    A = [k for k in range(d) if k % 2 == layer % 2]
    B = [k for k in range(d) if k % 2 != layer % 2]
    return A, B


def layer_sizes(d, layer, H=HIDDEN):
    A, B = masks(d, layer)
    a, b = len(A), len(B)
    return [("W1", (H, a)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (2 * b, H)), ("b3", (2 * b,))]


def param_count(d, H=HIDDEN):
    return sum(int(np.prod(shape)) for l in range(LAYERS) for _, shape in layer_sizes(d, l, H))


def unpack(theta, d, H=HIDDEN):
    """views of the flat vector as the per-layer arrays"""
    out, off = [], 0
    for l in range(LAYERS):
        layer = {}
        for name, shape in layer_sizes(d, l, H):
            n = int(np.prod(shape))
            layer[name] = theta[off:off + n].reshape(shape)
            off += n
        out.append(layer)
    assert off == theta.size
    return out


def bf16(a):
    """round to bf16 (nearest, ties to even) via the FP32 value, returned as float64"""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _log_sig_prime(z):
    az = np.abs(z)
    return -az - 2.0 * np.log1p(np.exp(-az))


def _logit(x):
    with np.errstate(divide="ignore"):
        return np.clip(np.log(x) - np.log1p(-x), -Z_CLAMP, Z_CLAMP)


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def _mlp(layer, h, rnd):
    """conditioner of one layer on a batch h [n][a]: (s, t, cache)"""
    W1, W2, W3 = (rnd(layer[k]) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (layer[k] for k in ("b1", "b2", "b3"))  # biases stay FP32 values
    hq = rnd(h)
    a1 = hq @ W1.T + b1
    u1 = rnd(np.maximum(a1, 0.0))
    a2 = u1 @ W2.T + b2
    u2 = rnd(np.maximum(a2, 0.0))
    o = u2 @ W3.T + b3
    s = S_CLAMP * np.tanh(o[:, 0::2] / S_CLAMP)
    t = o[:, 1::2]
    return s, t, (hq, a1, u1, a2, u2, W1, W2, W3)


def _ident(a):
    return np.asarray(a, dtype=np.float64)


def normalise(theta, x, d, bf16_path=False, keep=False):
    """N: x [n][d] -> (x' [n][d], log|det dN/dx| [n]); keep=True also returns the layer caches"""
    rnd = bf16 if bf16_path else _ident
    layers = unpack(np.asarray(theta, dtype=np.float64), d)
    z = _logit(np.asarray(x, dtype=np.float64))
    logdet = -_log_sig_prime(z).sum(axis=1)
    caches = []
    for l in range(LAYERS):
        A, B = masks(d, l)
        s, t, cache = _mlp(layers[l], z[:, A], rnd)
        zin = z[:, B].copy()
        z[:, B] = zin * np.exp(s) + t
        logdet += s.sum(axis=1)
        caches.append((A, B, s, zin, cache))
    logdet += _log_sig_prime(z).sum(axis=1)
    xp = _sigmoid(z)
    if keep:
        return xp, logdet, z, caches
    return xp, logdet


def sample(theta, xp, d, bf16_path=False):
    """F = N^-1: x' [n][d] -> (x [n][d], log|det dF/dx'| [n])"""
    rnd = bf16 if bf16_path else _ident
    layers = unpack(np.asarray(theta, dtype=np.float64), d)
    z = _logit(np.asarray(xp, dtype=np.float64))
    logdet = -_log_sig_prime(z).sum(axis=1)
    for l in reversed(range(LAYERS)):
        A, B = masks(d, l)
        s, t, _ = _mlp(layers[l], z[:, A], rnd)
        z[:, B] = (z[:, B] - t) * np.exp(-s)
        logdet -= s.sum(axis=1)
    logdet += _log_sig_prime(z).sum(axis=1)
    return _sigmoid(z), logdet


def loss(theta, x, w, d, bf16_path=False):
    """- sum w log q(x) / sum w, q the flow's density of x with a uniform base"""
    _, logdet = normalise(theta, x, d, bf16_path)
    w = np.asarray(w, dtype=np.float64)
    return -float(np.dot(w, logdet) / w.sum())


def grad(theta, x, w, d, bf16_path=False, bf16_grad=False):
    """(loss, d loss / d theta) by backpropagation through N.  bf16_grad=True also rounds to bf16 what the
    tensor-core gradient stores as bf16 operands: the gradient of the coupling outputs (s, t) and of the two
    hidden pre-activations after the ReLU mask; the weight and bias gradients are then sums over those rounded
    values"""
    theta = np.asarray(theta, dtype=np.float64)
    gq = bf16 if bf16_grad else _ident
    w = np.asarray(w, dtype=np.float64)
    wn = w / w.sum()
    xp, logdet, z, caches = normalise(theta, x, d, bf16_path, keep=True)
    L = -float(np.dot(wn, logdet))
    g = np.zeros_like(theta)
    gl = unpack(g, d)
    # d loss / d z after the last layer, from the output wrap term sum_k ls(z_k)
    gz = -wn[:, None] * (1.0 - 2.0 * _sigmoid(z))
    for l in reversed(range(LAYERS)):
        A, B, s, zin, (hq, a1, u1, a2, u2, W1, W2, W3) = caches[l]
        gzB = gz[:, B]
        es = np.exp(s)
        gs = -wn[:, None] + gzB * zin * es   # the logdet term and z_out = z_in e^s + t
        gt = gzB
        go = np.empty((x.shape[0], 2 * len(B)))
        go[:, 0::2] = gs * (1.0 - (s / S_CLAMP) ** 2)
        go[:, 1::2] = gt
        go = gq(go)
        gl[l]["W3"][...] = go.T @ u2
        gl[l]["b3"][...] = go.sum(axis=0)
        gu2 = go @ W3
        ga2 = gq(gu2 * (a2 > 0.0))
        gl[l]["W2"][...] = ga2.T @ u1
        gl[l]["b2"][...] = ga2.sum(axis=0)
        gu1 = ga2 @ W2
        ga1 = gq(gu1 * (a1 > 0.0))
        gl[l]["W1"][...] = ga1.T @ hq
        gl[l]["b1"][...] = ga1.sum(axis=0)
        gh = ga1 @ W1
        gz_new = gz.copy()
        gz_new[:, B] = gzB * es
        gz_new[:, A] += gh
        gz = gz_new
    return L, g


def adam(theta, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """one Adam update (Kingma and Ba, Algorithm 1); step counts from 1; returns (theta, m, v)"""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
