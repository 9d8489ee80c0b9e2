"""MLP surrogate on the GPU (tensor-core BF16 kernels) against the FP64 MLP oracle.

Tolerance for network outputs (derived from the arithmetic, not fitted).  The kernels round
the inputs, the weights and every stored activation / tangent tile to BF16 (8 significant
bits: unit roundoff u = 2^-8) and accumulate in FP32 (error negligible against u); biases,
the SiLU evaluation and the first tangent seed W1 are FP32.  Two first-order propagations of
those roundings through the network are evaluated in FP64 from the oracle's own forward pass:

* worst case: every rounding at its bound u|t| with the signs aligned (absolute values);
* probabilistic: every rounding an independent zero-mean error of variance at most u^2 t^2 / 3
  (round to nearest errs by at most half an ulp, <= u|t|, modelled as uniform), variances
  added through the layers (the sqrt(n) growth of probabilistic rounding-error analysis, as
  opposed to the n growth of the worst case; where two error terms share sources their
  variances are added with a factor 2, the bound for correlated terms).

The tests allow min(6 sigma, worst case) per sample and entry.  For networks of 64-wide layers
the worst case grows like (sum |W|)^layers and exceeds the outputs themselves; the 6-sigma
bound is the informative one.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_2604_22087_b300 import inputs as I

pytestmark = pytest.mark.gpu
U = 2.0 ** -8  # BF16 unit roundoff (8 significant bits)
K_SIGMA = 6.0


def J():
    from paper_2604_22087_b300 import jetsci
    return jetsci


def config(range_=0.05):
    # per-phase output scale: Young's modulus times the strain range, zero shift
    sc = np.array([[I.MATRIX_E * range_] * 6, [I.INCLUSION_E * range_] * 6])
    return dict(in_scale=range_, range_=range_, out_scale=sc, out_shift=np.zeros((2, 6)))


def silu_pp(z):
    """silu''(z) = s (1 - s) (2 + z (1 - 2 s)), s = sigmoid(z); |silu''| <= 0.5."""
    s = mlp.sigmoid(z)
    return s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s))


def forward_bound(layers, x):
    """Worst-case first-order bound on |y_bf16 - y| per sample and output."""
    _, zs, acts = mlp.forward(layers, x, keep=True)
    absW = [np.abs(W) for W, _ in layers]
    da = U * np.abs(x)
    for li in range(3):
        dz = da @ absW[li].T + U * (np.abs(acts[li]) @ absW[li].T)
        da = np.abs(mlp.silu_prime(zs[li])) * dz + U * np.abs(acts[li + 1])
    return da @ absW[3].T + U * (np.abs(acts[3]) @ absW[3].T)


def forward_sigma(layers, x):
    """Standard deviation of y_bf16 - y per sample and output under independent roundings."""
    _, zs, acts = mlp.forward(layers, x, keep=True)
    W2 = [W * W for W, _ in layers]
    r = U * U / 3.0
    va = r * x * x
    for li in range(3):
        vz = va @ W2[li].T + r * ((acts[li] ** 2) @ W2[li].T)
        va = mlp.silu_prime(zs[li]) ** 2 * vz + r * acts[li + 1] ** 2
    return np.sqrt(va @ W2[3].T + r * ((acts[3] ** 2) @ W2[3].T))


def _zsigma(layers, x):
    """Variances of the errors of z_1..z_3 (for the silu' factors of the tangent pass)."""
    _, zs, acts = mlp.forward(layers, x, keep=True)
    W2 = [W * W for W, _ in layers]
    r = U * U / 3.0
    va = r * x * x
    out = []
    for li in range(3):
        vz = va @ W2[li].T + r * ((acts[li] ** 2) @ W2[li].T)
        out.append(vz)
        va = mlp.silu_prime(zs[li]) ** 2 * vz + r * acts[li + 1] ** 2
    return zs, out


def jacobian_bound(layers, x):
    """Worst-case first-order bound on the input-Jacobian rows (per sample, output, direction)."""
    _, zs, acts = mlp.forward(layers, x, keep=True)
    absW = [np.abs(W) for W, _ in layers]
    da = U * np.abs(x)
    dzs = []
    for li in range(3):
        dz = da @ absW[li].T + U * (np.abs(acts[li]) @ absW[li].T)
        dzs.append(dz)
        da = np.abs(mlp.silu_prime(zs[li])) * dz + U * np.abs(acts[li + 1])
    W1 = layers[0][0][:, :6]
    T = mlp.silu_prime(zs[0])[:, :, None] * W1[None]            # [n, 64, 6]
    dT = (np.abs(silu_pp(zs[0])) * dzs[0])[:, :, None] * np.abs(W1)[None] + U * np.abs(T)
    for li in (1, 2):
        W = layers[li][0]
        V = np.einsum("oh,nhd->nod", W, T)
        dV = np.einsum("oh,nhd->nod", absW[li], dT) + U * np.einsum("oh,nhd->nod", absW[li], np.abs(T))
        sp = mlp.silu_prime(zs[li])[:, :, None]
        T = sp * V
        dT = np.abs(sp) * dV + (np.abs(silu_pp(zs[li])) * dzs[li])[:, :, None] * np.abs(V) + U * np.abs(T)
    return np.einsum("oh,nhd->nod", absW[3], dT) + U * np.einsum("oh,nhd->nod", absW[3], np.abs(T))


def jacobian_sigma(layers, x):
    """Standard deviation of the input-Jacobian error under independent roundings."""
    zs, vzs = _zsigma(layers, x)
    W2 = [W * W for W, _ in layers]
    r = U * U / 3.0
    W1 = layers[0][0][:, :6]
    T = mlp.silu_prime(zs[0])[:, :, None] * W1[None]
    # T1 = silu'(z1) W1 (FP32 seed), rounded to BF16; silu'(z1) carries z1's error
    vT = (silu_pp(zs[0]) ** 2 * vzs[0])[:, :, None] * (W1 * W1)[None] + r * T * T
    for li in (1, 2):
        W = layers[li][0]
        V = np.einsum("oh,nhd->nod", W, T)
        vV = np.einsum("oh,nhd->nod", W2[li], vT) + r * np.einsum("oh,nhd->nod", W2[li], T * T)
        sp = mlp.silu_prime(zs[li])[:, :, None]
        T = sp * V
        # the two terms share error sources: variances added with a factor 2
        vT = 2.0 * (sp * sp * vV + (silu_pp(zs[li]) ** 2 * vzs[li])[:, :, None] * V * V) + r * T * T
    return np.sqrt(np.einsum("oh,nhd->nod", W2[3], vT) + r * np.einsum("oh,nhd->nod", W2[3], T * T))


def output_bounds(layers, x):
    """(|dy| bound [n, 6], |dJ| bound [n, 6, 6]): min(6 sigma, worst case) per entry."""
    by = np.minimum(K_SIGMA * forward_sigma(layers, x), forward_bound(layers, x))
    bJ = np.minimum(K_SIGMA * jacobian_sigma(layers, x), jacobian_bound(layers, x))
    return by, bJ


def nh_stress_oracle(E6, phase):
    """S(E) of the oracle's neo-Hookean law, via any F with F^T F = I + 2E."""
    out = np.zeros_like(E6)
    lm = [oracle.lame(I.MATRIX_E, I.MATRIX_NU), oracle.lame(I.INCLUSION_E, I.INCLUSION_NU)]
    for i in range(len(E6)):
        e = E6[i]
        E = np.array([[e[0], e[5], e[4]], [e[5], e[1], e[3]], [e[4], e[3], e[2]]])
        L = np.linalg.cholesky(np.eye(3) + 2 * E)
        S, _ = oracle.neo_hookean(*lm[phase[i]], L.T)
        out[i] = [S[0, 0], S[1, 1], S[2, 2], S[1, 2], S[0, 2], S[0, 1]]
    return out


@pytest.fixture(scope="module")
def data():
    E6, ph = I.strain_samples(4096, seed=11)
    return E6, ph, torch.as_tensor(E6).cuda(), torch.as_tensor(ph).cuda()


def test_labels_match_oracle_neo_hookean(data):
    E6, ph, E6d, phd = data
    S = J().Surrogate.label(I.composite_materials(I.LAW_NEO_HOOKEAN), E6d, phd).cpu().numpy()
    ref = nh_stress_oracle(E6[:512], ph[:512])
    assert np.max(np.abs(S[:512] - ref)) <= 1e-13 * np.max(np.abs(ref))


def _layers(seed):
    g = np.random.default_rng(seed)
    return [(W, g.uniform(-0.1, 0.1, b.shape)) for W, b in I.mlp_init(seed)]


def test_eval_and_input_jacobian_within_bf16_bound(data):
    E6, ph, E6d, phd = data
    cfg = config()
    s = J().Surrogate(_layers(3), **cfg)
    layers = s.layers()  # FP32 master weights as the oracle sees them
    S, D = s.eval(E6d, phd)
    S, D = S.cpu().numpy(), D.cpu().numpy()
    x = mlp.surrogate_inputs(E6, ph, cfg["in_scale"])
    y_ref = mlp.forward(layers, x)
    sc = cfg["out_scale"][ph]
    y_gpu = S / sc
    bound, jb = output_bounds(layers, x)
    # the bounds are informative: well below the outputs they bound
    assert np.max(bound) <= 0.05 * np.max(np.abs(y_ref))
    assert np.all(np.abs(y_gpu - y_ref) <= bound + 1e-6)
    Jm_ref = mlp.input_jacobian(layers, x)
    Jm_gpu = D * cfg["in_scale"] / sc[:, :, None]
    assert np.max(jb) <= 0.05 * np.max(np.abs(Jm_ref))
    assert np.all(np.abs(Jm_gpu - Jm_ref) <= jb + 1e-6)
    # and the oracle's own surrogate map agrees on S and D up to the same bounds
    S_o, D_o = mlp.surrogate_stress(layers, E6, ph, cfg["in_scale"], cfg["out_scale"], cfg["out_shift"])
    assert np.all(np.abs(S - S_o) <= (bound + 1e-6) * sc)


def test_minibatch_gradient_matches_oracle_reverse_mode(data):
    E6, ph, E6d, phd = data
    cfg = config()
    mats = I.composite_materials(I.LAW_NEO_HOOKEAN)
    Sd = J().Surrogate.label(mats, E6d, phd)
    s = J().Surrogate(_layers(5), **cfg)
    batch = 1024
    order = torch.arange(batch, dtype=torch.int32, device="cuda")
    grad, loss = s.gradient(E6d, phd, Sd, order, batch)
    layers = s.layers()
    x = mlp.surrogate_inputs(E6[:batch], ph[:batch], cfg["in_scale"])
    t = (Sd.cpu().numpy()[:batch] - cfg["out_shift"][ph[:batch]]) / cfg["out_scale"][ph[:batch]]
    loss_ref, grads_ref = mlp.gradients(layers, x, t)
    g_ref = J().pack_layers(grads_ref)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - loss_ref) <= 2e-2 * loss_ref
    # per layer, normwise: 4 layers x 2 BF16 roundings x u ~ 1.6e-2
    offs = [0, 512, 576, 4672, 4736, 8832, 8896, 9280, 9286]
    for a, b in zip(offs[:-1], offs[1:]):
        assert np.max(np.abs(g[a:b] - g_ref[a:b])) <= 2e-2 * np.max(np.abs(g_ref[a:b])), (a, b)


def test_adam_first_step_on_device(data):
    E6, ph, E6d, phd = data
    cfg = config()
    Sd = J().Surrogate.label(I.composite_materials(I.LAW_NEO_HOOKEAN), E6d, phd)
    s = J().Surrogate(_layers(6), **cfg)
    order = torch.arange(512, dtype=torch.int32, device="cuda")
    grad, _ = s.gradient(E6d, phd, Sd, order, 512)
    p0 = s.params()
    s.train(E6d, phd, Sd, order, n_steps=1, batch=512, lr_max=1e-3, lr_min=1e-3)
    p1 = s.params()
    g = grad.cpu().numpy().astype(np.float64)
    expect = p0 - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(p1 - expect)) <= 1e-3 * 1e-4 + 1e-7 * np.max(np.abs(p0))


def test_checkpoint_round_trip(data, tmp_path):
    """save() then load() restores the weights and scalings: the restored surrogate evaluates
    S and D bit for bit like the original, and metadata given to save() is kept."""
    E6, ph, E6d, phd = data
    s = J().Surrogate(_layers(7), **config())
    path = tmp_path / "surrogate.npz"
    s.save(path, seed=7)
    t = J().Surrogate.load(path)
    assert np.array_equal(s.params(), t.params())
    S1, D1 = s.eval(E6d, phd)
    S2, D2 = t.eval(E6d, phd)
    assert torch.equal(S1, S2) and torch.equal(D1, D2)
    assert int(np.load(path)["seed"]) == 7
    s.close()
    t.close()


def test_training_learns_the_neo_hookean_law():
    """Train on NH labels with the library's kernels: the trained network is far closer to the
    plain neo-Hookean law than the untrained network and than small-strain Hooke with the same
    Lame constants (the cheaper law it could otherwise stand in for).  This is what training
    gains; it is not a gain over the neo-Hookean update itself, which is exact by definition
    and, evaluated in FP32 on this GPU, cheaper per Gauss point than the network's forward
    pass."""
    n = 1 << 16
    E6, ph = I.strain_samples(n, seed=5)
    E6d, phd = torch.as_tensor(E6).cuda(), torch.as_tensor(ph).cuda()
    mats = I.composite_materials(I.LAW_NEO_HOOKEAN)
    Sd = J().Surrogate.label(mats, E6d, phd)
    cfg = config()
    s = J().Surrogate(I.mlp_init(5), **cfg)
    Et, pt = I.strain_samples(2048, seed=99)
    Etd, ptd = torch.as_tensor(Et).cuda(), torch.as_tensor(pt).cuda()
    S_true = J().Surrogate.label(mats, Etd, ptd).cpu().numpy()
    scale = cfg["out_scale"][pt]

    def err(S):
        return float(np.sqrt(np.mean(((S - S_true) / scale) ** 2)))

    e0 = err(s.eval(Etd, ptd, tangent=False).cpu().numpy())
    epochs, batch = 20, 2048
    order = torch.as_tensor(I.minibatch_order(n, epochs, seed=5)).cuda()
    steps = epochs * (n // batch)
    losses = s.train(E6d, phd, Sd, order, n_steps=steps, batch=batch, lr_max=3e-3, lr_min=1e-5).cpu().numpy()
    e1 = err(s.eval(Etd, ptd, tangent=False).cpu().numpy())
    # small-strain Hooke with the same Lame constants (the method without the learned law)
    hooke = np.zeros_like(S_true)
    for p, (E, nu, _) in enumerate(mats):
        lam, mu = oracle.lame(E, nu)
        m = pt == p
        tr = Et[m, :3].sum(1)
        hooke[m, :3] = lam * tr[:, None] + 2 * mu * Et[m, :3]
        hooke[m, 3:] = 2 * mu * Et[m, 3:]
    e_hooke = err(hooke)
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.02 * losses[:50].mean()
    assert e1 < 0.05 * e0
    assert e1 < 0.2 * e_hooke, (e1, e_hooke)
