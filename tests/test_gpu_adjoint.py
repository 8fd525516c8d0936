"""GPU adjoint gradient of the final energy density with respect to the
per-period kick angles and drive fields, through the C ABI: against the
FP64 oracle's adjoint (itself pinned by finite differences on the CPU) and
against central finite differences of the GPU's own evolution."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import capi, inputs

pytestmark = pytest.mark.gpu


def _cfg(L, P, seed, first_layer=0, ew=0.5):
    rng = np.random.default_rng(seed)
    return inputs.ChainConfig(L=L, periods=P, seed=seed, first_layer=first_layer,
                              edge_field_weight=ew, theta_p=rng.uniform(0.1, 0.5, P),
                              hx_p=rng.uniform(0.6, 1.0, P))


def _gpu_adjoint(cfg, precision):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    with FloquetSimulator(cfg.L, precision=precision) as sim:
        sim.init_product_state(cfg.spinors())
        psi0 = sim.host_state()
        sim.build(**chain_params(cfg))
        gt, gh, e = sim.adjoint()
        psi1 = sim.host_state()
        assert sim.period == 0
    return gt, gh, e, psi0, psi1


def _oracle_adjoint(cfg):
    hdrive, hobs = orc.chain_inputs(cfg)
    dh = np.stack([orc.ising_dh_dhx(cfg.L, cfg.edge_field_weight)] * cfg.periods)
    psi = orc.product_state(cfg.spinors())
    return orc.adjoint(psi, hdrive, dh, cfg.tau, cfg.theta_p, cfg.K, cfg.first_layer, hobs)


def _gpu_final_energy(cfg, theta_p, hx_p, precision="c128"):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    c = inputs.ChainConfig(L=cfg.L, periods=cfg.periods, seed=cfg.seed,
                           first_layer=cfg.first_layer, edge_field_weight=cfg.edge_field_weight,
                           theta_p=theta_p, hx_p=hx_p)
    with FloquetSimulator(c.L, precision=precision) as sim:
        sim.init_product_state(c.spinors())
        sim.build(**chain_params(c))
        e, _ = sim.evolve(c.periods)
    return e[-1]


@pytest.mark.parametrize("L,P,first,ew", [(6, 3, 0, 0.5), (9, 4, 1, 1.0), (10, 5, 0, 0.5)])
def test_adjoint_c128_matches_oracle(svlib, L, P, first, ew):
    cfg = _cfg(L, P, seed=10 + L, first_layer=first, ew=ew)
    gt, gh, e, psi0, psi1 = _gpu_adjoint(cfg, "c128")
    ot, oh, oe = _oracle_adjoint(cfg)
    assert abs(e - oe) < 1e-12
    np.testing.assert_allclose(gt, ot, atol=1e-11, rtol=1e-10)
    np.testing.assert_allclose(gh, oh, atol=1e-11, rtol=1e-10)
    # the reverse sweep hands back the starting state
    assert np.linalg.norm(psi1 - psi0) < 1e-11


@pytest.mark.parametrize("L,P", [(10, 5), (14, 6)])
def test_adjoint_c64_matches_oracle(svlib, L, P):
    cfg = _cfg(L, P, seed=20 + L)
    gt, gh, e, psi0, psi1 = _gpu_adjoint(cfg, "c64")
    ot, oh, oe = _oracle_adjoint(cfg)
    assert abs(e - oe) < 1e-5
    scale = max(np.abs(ot).max(), np.abs(oh).max())
    np.testing.assert_allclose(gt, ot, atol=1e-4 * scale, rtol=0)
    np.testing.assert_allclose(gh, oh, atol=1e-4 * scale, rtol=0)
    assert np.linalg.norm(psi1.astype(np.complex128) - psi0) < 1e-4


def test_adjoint_matches_gpu_finite_differences(svlib):
    """Central differences of the complex128 GPU evolution, per parameter."""
    cfg = _cfg(12, 4, seed=33)
    gt, gh, e, _, _ = _gpu_adjoint(cfg, "c128")
    eps = 1e-4
    for p in range(cfg.periods):
        d = np.zeros(cfg.periods)
        d[p] = eps
        fd_t = (_gpu_final_energy(cfg, cfg.theta_p + d, cfg.hx_p)
                - _gpu_final_energy(cfg, cfg.theta_p - d, cfg.hx_p)) / (2 * eps)
        fd_h = (_gpu_final_energy(cfg, cfg.theta_p, cfg.hx_p + d)
                - _gpu_final_energy(cfg, cfg.theta_p, cfg.hx_p - d)) / (2 * eps)
        # O(eps^2) truncation of the central difference
        assert abs(gt[p] - fd_t) < 1e-7 * max(1.0, abs(fd_t)), (p, gt[p], fd_t)
        assert abs(gh[p] - fd_h) < 1e-7 * max(1.0, abs(fd_h)), (p, gh[p], fd_h)


def test_adjoint_L20_200_periods_directional(svlib):
    """L=20, 200 periods, 400 parameters: the directional derivative along a
    random unit vector against a central difference of the complex128 GPU
    evolution (step 1e-3), and the complex64 gradient against the
    complex128 one."""
    P = 200
    cfg = _cfg(20, P, seed=3)
    cfg.theta_p[:] = 0.3
    cfg.hx_p[:] = 0.9
    gt, gh, e, _, _ = _gpu_adjoint(cfg, "c128")
    rng = np.random.default_rng(7)
    v = rng.standard_normal(2 * P)
    v /= np.linalg.norm(v)
    vt, vh = v[:P], v[P:]
    eps = 1e-3
    fd = (_gpu_final_energy(cfg, cfg.theta_p + eps * vt, cfg.hx_p + eps * vh)
          - _gpu_final_energy(cfg, cfg.theta_p - eps * vt, cfg.hx_p - eps * vh)) / (2 * eps)
    ad = float(gt @ vt + gh @ vh)
    assert abs(ad - fd) < 1e-4 * max(abs(fd), 1e-3), (ad, fd)
    gt32, gh32, e32, _, _ = _gpu_adjoint(cfg, "c64")
    assert abs(e32 - e) < 1e-5
    scale = max(np.abs(gt).max(), np.abs(gh).max())
    assert np.abs(gt32 - gt).max() < 1e-3 * scale
    assert np.abs(gh32 - gh).max() < 1e-3 * scale


def test_adjoint_over_fewer_periods_than_parameters(svlib):
    """sv_adjoint(periods = P' < n_period_params) differentiates the energy
    after P' periods: the oracle's adjoint of the first P' periods."""
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = _cfg(8, 5, seed=21)
    with FloquetSimulator(cfg.L, precision="c128") as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**chain_params(cfg))
        gt, gh, e = sim.adjoint(periods=3)
        for bad in (0, 6):
            with pytest.raises(capi.SvError) as ei:
                sim.adjoint(periods=bad)
            assert ei.value.code == capi.SV_EINVAL
    short = inputs.ChainConfig(L=cfg.L, periods=3, seed=cfg.seed, first_layer=cfg.first_layer,
                               edge_field_weight=cfg.edge_field_weight,
                               theta_p=cfg.theta_p[:3], hx_p=cfg.hx_p[:3])
    ot, oh, oe = _oracle_adjoint(short)
    assert gt.shape == (3,) and abs(e - oe) < 1e-12
    np.testing.assert_allclose(gt, ot, atol=1e-11, rtol=1e-10)
    np.testing.assert_allclose(gh, oh, atol=1e-11, rtol=1e-10)


def test_adjoint_call_order(svlib):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = _cfg(8, 3, seed=1)
    with FloquetSimulator(cfg.L) as sim:
        sim.init_product_state(cfg.spinors())
        plain = inputs.ChainConfig(L=8, seed=1)
        sim.build(**chain_params(plain))
        with pytest.raises(capi.SvError) as ei:
            sim.adjoint()
        assert ei.value.code == capi.SV_ESTATE  # no per-period parameters
        sim.build(**chain_params(cfg))
        sim.evolve(1)
        with pytest.raises(capi.SvError) as ei:
            sim.adjoint()
        assert ei.value.code == capi.SV_ESTATE  # not at period 0


def test_autograd_function_gradcheck(svlib):
    import torch
    from paper_2111_08044_gb300.autograd import final_energy
    cfg = inputs.ChainConfig(L=8, periods=3, seed=4)
    rng = np.random.default_rng(4)
    th = torch.tensor(rng.uniform(0.1, 0.5, 3), dtype=torch.float64, requires_grad=True)
    hx = torch.tensor(rng.uniform(0.6, 1.0, 3), dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda a, b: final_energy(a, b, cfg, "c128"), (th, hx),
                                    eps=1e-6, atol=1e-7, rtol=1e-5)
    e = final_energy(th, hx, cfg, "c128")
    e.backward()
    ot, oh, oe = _oracle_adjoint(inputs.ChainConfig(L=8, periods=3, seed=4,
                                                    theta_p=th.detach().numpy(),
                                                    hx_p=hx.detach().numpy()))
    assert abs(float(e.detach()) - oe) < 1e-12
    np.testing.assert_allclose(th.grad.numpy(), ot, atol=1e-11, rtol=1e-10)
    np.testing.assert_allclose(hx.grad.numpy(), oh, atol=1e-11, rtol=1e-10)
