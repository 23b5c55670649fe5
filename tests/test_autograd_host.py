"""Host-side wiring of the differentiation layers, on the CPU: the library calls are replaced by
an analytic toy forward model with a known Hessian, M(C) = A (C * C) per map (A a fixed matrix),
so that what is checked is the plumbing. That means which product each autograd node returns,
the double-backward composition, chunking, and the unit scaling of the directions handed to the
Hessian-vector products. The kernels themselves are checked against the oracle in the GPU tests.

Toy model: J = dM/dC = A diag(2C), J^T w = 2C * (A^T w), d/dC[J^T w] . v = 2v * (A^T w)."""
import numpy as np
import pytest
import torch

from paper_2603_04070_gb300 import autograd, fwi, unfolded

NZ, NX, M_OUT = 3, 4, 7


class Toy:
    def __init__(self, seed=0):
        g = torch.Generator().manual_seed(seed)
        self.A = torch.randn(M_OUT, NZ * NX, generator=g, dtype=torch.float64)
        self.calls = {"hvp": [], "second_order": []}

    def F(self, c):
        return (c.reshape(c.shape[0], -1) ** 2) @ self.A.T          # [B, M_OUT]

    def JTw(self, c, w):
        return (2.0 * c.reshape(c.shape[0], -1) * (w @ self.A)).reshape(c.shape)

    # the binding's signatures, as the wrappers call them
    def forward_save(self, problem, sos, wavelet, geom, **kw):
        return self.F(sos).reshape(sos.shape[0], 1, M_OUT, 1), "ws"

    def backward(self, problem, sos, wavelet, geom, cd_grad, ws, **kw):
        return self.JTw(sos, cd_grad.reshape(sos.shape[0], M_OUT))

    def jvp(self, problem, sos, wavelet, geom, v, **kw):
        c = sos.reshape(sos.shape[0], -1)
        return ((2.0 * c * v.reshape(c.shape)) @ self.A.T).reshape(sos.shape[0], 1, M_OUT, 1)

    def second_order(self, problem, sos, wavelet, geom, cd_grad, v, **kw):
        self.calls["second_order"].append(float(v.abs().max()))
        w = cd_grad.reshape(sos.shape[0], M_OUT)
        so = (2.0 * v.reshape(sos.shape[0], -1) * (w @ self.A)).reshape(sos.shape)
        return so, self.jvp(problem, sos, wavelet, geom, v)

    def misfit_gradient(self, problem, sos, wavelet, geom, cd_obs, **kw):
        r = self.F(sos) - cd_obs.reshape(sos.shape[0], M_OUT)
        return (r * r).sum(1), self.JTw(sos, 2.0 * r)

    def hvp(self, problem, sos, wavelet, geom, cd_obs, v, **kw):
        self.calls["hvp"].append(float(v.abs().max()))
        r = self.F(sos) - cd_obs.reshape(sos.shape[0], M_OUT)
        Jv = (2.0 * sos.reshape(sos.shape[0], -1) * v.reshape(sos.shape[0], -1)) @ self.A.T
        return self.JTw(sos, 2.0 * Jv) + (2.0 * v.reshape(sos.shape[0], -1) * ((2.0 * r) @ self.A)).reshape(sos.shape)

    def dense_hessian(self, c, obs):
        """Per map: H = 2 J^T J + diag(2 A^T w), w = 2 (M - M_obs)."""
        Hs = []
        for b in range(c.shape[0]):
            cb = c[b].reshape(-1)
            Jb = self.A * (2.0 * cb)[None, :]
            r = (cb ** 2) @ self.A.T - obs[b].reshape(-1)
            Hs.append(2.0 * Jb.T @ Jb + torch.diag(2.0 * ((2.0 * r) @ self.A)))
        return Hs


@pytest.fixture
def toy(monkeypatch):
    t = Toy()
    for name in ("forward_save", "backward", "jvp", "second_order", "misfit_gradient", "hvp"):
        monkeypatch.setattr(autograd.dufwi, name, getattr(t, name))
    return t


def _case(B=3, seed=1):
    g = torch.Generator().manual_seed(seed)
    c = 1.0 + 0.5 * torch.rand(B, NZ, NX, generator=g, dtype=torch.float64)
    obs = torch.randn(B, 1, M_OUT, 1, generator=g, dtype=torch.float64)
    v = torch.randn(B, NZ, NX, generator=g, dtype=torch.float64)
    return c, obs, v


def test_double_backward_gives_the_exact_hessian(toy):
    c, obs, v = _case()
    Hv = autograd.hvp(None, c, torch.zeros(1), None, obs, v)
    for b, H in enumerate(toy.dense_hessian(c, obs)):
        assert torch.allclose(Hv[b].reshape(-1), H @ v[b].reshape(-1), rtol=1e-12, atol=1e-12)


def test_first_backward_without_graph_is_the_plain_vjp(toy):
    c, obs, v = _case()
    x = c.clone().requires_grad_(True)
    J = autograd.misfit(None, x, torch.zeros(1), None, obs).sum()
    (g,) = torch.autograd.grad(J, x)
    _, g_ref = toy.misfit_gradient(None, c, None, None, obs)
    assert torch.allclose(g, g_ref, rtol=1e-12)
    assert toy.calls["second_order"] == []


def test_data_gradient_node_backward_is_hessian_for_any_cotangent_scale(toy):
    """The unfolded loop's g = dJ/dC node: backward applies H, with the direction handed to the
    HVP scaled to unit max-norm per map whatever the cotangent's scale, across chunk sizes."""
    c, obs, _ = _case(B=5)
    phys = unfolded.Physics(None, torch.zeros(1), None)
    Hs = toy.dense_hessian(c, obs)
    for scale in (1e-17, 1.0, 1e6):
        for chunk in (1, 2, 8):
            toy.calls["hvp"].clear()
            x = c.clone().requires_grad_(True)
            g = unfolded.data_gradient_differentiable(phys, x, obs, chunk=chunk)
            gbar = scale * torch.randn(c.shape, dtype=torch.float64)
            (Hg,) = torch.autograd.grad(g, x, grad_outputs=gbar)
            for b, H in enumerate(Hs):
                ref = H @ gbar[b].reshape(-1)
                assert torch.allclose(Hg[b].reshape(-1), ref, rtol=1e-10, atol=1e-12 * float(ref.abs().max()))
            assert len(toy.calls["hvp"]) == -(-5 // chunk)
            assert all(abs(m - 1.0) < 1e-12 for m in toy.calls["hvp"])


def test_newton_cg_hessvec_calls_use_unit_scaled_directions(toy):
    """Truncated Newton on the toy misfit: every Hessian-vector product it requests has unit
    max-norm directions, and it lowers the misfit."""
    c, obs, _ = _case(B=2, seed=3)
    evaluate = lambda s, need: toy.misfit_gradient(None, s, None, None, obs) if need else \
        (toy.misfit_gradient(None, s, None, None, obs)[0], None)
    hessvec = lambda s, v: toy.hvp(None, s, None, None, obs, v)
    toy.calls["hvp"].clear()
    res = fwi.newton_cg(evaluate, hessvec, c, 4, cg_iters=6, c_lo=-1e9, c_hi=1e9, sync=False)
    J = torch.stack(res.misfits)
    assert torch.all(J[1:] <= J[:-1])
    assert toy.calls["hvp"] and all(abs(m - 1.0) < 1e-12 for m in toy.calls["hvp"])
