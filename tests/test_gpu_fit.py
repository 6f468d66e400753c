"""Reverse mode of relight + projection (hand-written adjoint kernels behind torch.autograd) and
material fitting by Adam, checked against the FP64 oracle's hand gradient and central differences.

Coordinates of the fit: theta = (ln sigma_a[3], ln sigma_s'[3], eta, l[J]); loss
L = sum_{c,o} (B - B*)^2 with B* rendered from a hidden material.  Keep-all compression
(p = 1) makes the compressed transfer identical on both sides, so the only
differences are FP32 arithmetic on the GPU.
"""
import numpy as np
import pytest

from oracle import tsr_oracle as O
from paper_2203_12339_gb300 import scene

pytestmark = pytest.mark.gpu

NU, K, J = 16, 12, 16


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_12339_gb300 import build
    build.build()
    from paper_2203_12339_gb300 import tsr
    sa, ss = scene.pca_materials(256, seed=0)
    f, _ = O.fit_pca_basis(sa, ss, 1.3, 1024, 40.0, K)
    sc = scene.make_scene(NU, K=K, J=J, amp=0.1, seed=1)
    pos = sc.mesh.pos.astype(np.float32)
    area = sc.mesh.area.astype(np.float32)
    T = sc.T.astype(np.float32)
    M = O.transfer_full(f, pos, area, T)                 # FP64 oracle transfer
    Cw = O.chart_to_wavelet(M, NU)                       # keep-all compression
    basis = tsr.basis_create(f)
    comp = tsr.haar_compress(torch.tensor(M.astype(np.float32), device="cuda"), NU, 1.0)
    # hidden material (seed 3) and its target shading, all in FP64 on the oracle side
    rng = np.random.default_rng(3)
    h_sa = np.exp(rng.uniform(-7, 0, 3))
    h_ss = np.exp(rng.uniform(-1, 2, 3))
    h_eta = rng.uniform(1.2, 1.5)
    g_h = O.project_material(f, h_sa[None], h_ss[None], np.array([h_eta]))
    B_star = O.relight(Cw, NU, g_h, sc.light)
    return dict(torch=torch, tsr=tsr, f=f, Cw=Cw, basis=basis, comp=comp, light=sc.light, B_star=B_star)


def _oracle_loss(s, theta):
    sa = np.exp(theta[0:3])[None]
    ss = np.exp(theta[3:6])[None]
    eta = np.array([theta[6]])
    light = theta[7:]
    g = O.project_material(s["f"], sa, ss, eta)
    B = O.relight(s["Cw"], NU, g, light)
    return float(np.sum((B - s["B_star"]) ** 2))


def _oracle_grad(s, theta):
    sa = np.exp(theta[0:3])[None]
    ss = np.exp(theta[3:6])[None]
    eta = np.array([theta[6]])
    light = theta[7:]
    g = O.project_material(s["f"], sa, ss, eta)
    B = O.relight(s["Cw"], NU, g, light)
    dg, dl = O.relight_vjp(s["Cw"], NU, g, light, 2.0 * (B - s["B_star"]))
    d_sa, d_ss, d_eta = O.project_material_vjp(s["f"], sa, ss, eta, dg)
    return np.concatenate([d_sa[0] * sa[0], d_ss[0] * ss[0], d_eta, dl])   # chain rule to ln sigma


def _gpu_loss_grad(s, theta):
    torch, tsr = s["torch"], s["tsr"]
    from paper_2203_12339_gb300.autograd import render
    th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    sa = torch.exp(th[0:3]).reshape(1, 3)
    ss = torch.exp(th[3:6]).reshape(1, 3)
    eta = th[6:7]
    light = th[7:].float()
    B = render(s["comp"], s["basis"], sa, ss, eta, light)
    target = torch.tensor(s["B_star"], dtype=torch.float32, device="cuda")
    loss = ((B - target) ** 2).sum()
    loss.backward()
    tsr.stream_status()
    return float(loss), th.grad.cpu().numpy()


def _theta0():
    sa, ss, eta = scene.marble(1)
    light = scene.sh_light(J, 0)
    return np.concatenate([np.log(sa[0]), np.log(ss[0]), eta, light])


def _groups(v):
    return [v[0:3], v[3:6], v[6:7], v[7:]]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_oracle_gradient_matches_central_differences(setup):
    theta = _theta0()
    grad = _oracle_grad(setup, theta)
    h = 1e-4
    fd = np.empty_like(theta)
    for q in range(theta.size):
        tp = theta.copy()
        tm = theta.copy()
        tp[q] += h
        tm[q] -= h
        fd[q] = (_oracle_loss(setup, tp) - _oracle_loss(setup, tm)) / (2 * h)
    for a, b in zip(_groups(grad), _groups(fd)):
        assert _rel(a, b) <= 1e-4


def test_gpu_adjoint_matches_oracle_gradient_and_fd(setup):
    theta = _theta0()
    loss, grad = _gpu_loss_grad(setup, theta)
    assert loss == pytest.approx(_oracle_loss(setup, theta), rel=1e-5)
    ref = _oracle_grad(setup, theta)
    for a, b in zip(_groups(grad), _groups(ref)):
        assert _rel(a, b) <= 1e-4
    h = 1e-4
    for q in (0, 4, 6, 9):                  # spot FD checks of the GPU gradient (FP64 oracle forward)
        tp = theta.copy()
        tm = theta.copy()
        tp[q] += h
        tm[q] -= h
        fd = (_oracle_loss(setup, tp) - _oracle_loss(setup, tm)) / (2 * h)
        assert grad[q] == pytest.approx(fd, rel=1e-4, abs=1e-4 * np.abs(ref).max())


def test_adam_material_fit_reduces_loss(setup):
    torch = setup["torch"]
    from paper_2203_12339_gb300.autograd import render
    theta = torch.tensor(_theta0(), dtype=torch.float64, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([theta], lr=0.05, betas=(0.9, 0.999))
    target = torch.tensor(setup["B_star"], dtype=torch.float32, device="cuda")
    losses = []
    for _ in range(200):
        opt.zero_grad()
        sa = torch.exp(theta[0:3]).reshape(1, 3)
        ss = torch.exp(theta[3:6]).reshape(1, 3)
        eta = theta[6:7].clamp(1.0, 2.0)
        B = render(setup["comp"], setup["basis"], sa, ss, eta, theta[7:].float())
        loss = ((B - target) ** 2).sum()
        loss.backward()
        opt.step()
        with torch.no_grad():
            theta[6].clamp_(1.0, 2.0)
        losses.append(float(loss))
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 1e-2 * losses[0]


def test_gpu_adjoint_with_view_fresnel_matches_oracle(setup):
    """The same loss with the view-dependent Fresnel factor of Eq. 6 on the rendered shading: the eta
    gradient now also flows through dF_t/deta; GPU adjoint against the oracle's chain rule."""
    torch, tsr = setup["torch"], setup["tsr"]
    from paper_2203_12339_gb300.autograd import render
    N = 10 * NU * NU + 2
    cos_o = np.cos(np.linspace(0.0, 1.4, N))
    theta = _theta0()

    def oracle(theta):
        sa, ss = np.exp(theta[0:3])[None], np.exp(theta[3:6])[None]
        eta, light = np.array([theta[6]]), theta[7:]
        g = O.project_material(setup["f"], sa, ss, eta)
        B = O.relight(setup["Cw"], NU, g, light)
        Bv = O.fresnel_output(B, eta, cos_o)
        target = O.fresnel_output(setup["B_star"], np.array([1.35]), cos_o)
        loss = float(np.sum((Bv - target) ** 2))
        dBv = 2.0 * (Bv - target)
        dB, deta_f = O.fresnel_output_vjp(B, eta, cos_o, dBv)
        dg, dl = O.relight_vjp(setup["Cw"], NU, g, light, dB)
        d_sa, d_ss, d_eta = O.project_material_vjp(setup["f"], sa, ss, eta, dg)
        grad = np.concatenate([d_sa[0] * sa[0], d_ss[0] * ss[0], d_eta + deta_f, dl])
        return loss, grad, target

    loss_ref, grad_ref, target = oracle(theta)
    th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    B = render(setup["comp"], setup["basis"], torch.exp(th[0:3]).reshape(1, 3), torch.exp(th[3:6]).reshape(1, 3),
               th[6:7], th[7:].float(), torch.tensor(cos_o, dtype=torch.float32, device="cuda"))
    loss = ((B - torch.tensor(target, dtype=torch.float32, device="cuda")) ** 2).sum()
    loss.backward()
    tsr.stream_status()
    assert float(loss) == pytest.approx(loss_ref, rel=1e-5)
    grad = th.grad.cpu().numpy()
    for a, b in zip(_groups(grad), _groups(grad_ref)):
        assert _rel(a, b) <= 1e-4
    h = 1e-4   # and the oracle chain itself against central differences in eta
    tp, tm = theta.copy(), theta.copy()
    tp[6] += h
    tm[6] -= h
    fd = (oracle(tp)[0] - oracle(tm)[0]) / (2 * h)
    assert grad_ref[6] == pytest.approx(fd, rel=1e-4)
