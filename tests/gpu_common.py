"""Helpers shared by the GPU parity tests: one seeded system fed to both sides."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def make_pair(sysm, W, phi=None, dt=0.005, qr_period=5, seed=1, **kw):
    """A CUDA context and an oracle holding the same system and walkers."""
    from oracle.afqmc import Oracle
    from paper_2209_04015_b300 import AfqContext
    from paper_2209_04015_b300.synthetic import trial_walkers

    free = kw.pop("free_projection", False)
    cap = kw.pop("fb_cap", 0.0)
    order = kw.pop("taylor_order", 6)
    e_shift = kw.pop("e_shift", None)
    ctx = AfqContext(dt=dt, qr_period=qr_period, seed=seed, free_projection=free, fb_cap=cap,
                     taylor_order=order, e_shift=e_shift, **kw)
    ctx.init_hamiltonian(sysm.h1, sysm.L, sysm.e0)
    ctx.init_trial(sysm.psi_a, sysm.psi_b)
    phi0 = trial_walkers(sysm, W) if phi is None else phi
    ctx.init_walkers(W, phi0)
    orc = Oracle(sysm.h1, sysm.L, sysm.e0, sysm.psi_a, sysm.psi_b, dt=dt, qr_period=qr_period,
                 free_projection=free, fb_cap=cap, taylor_order=order, e_shift=e_shift)
    orc.init_walkers(phi0)
    return ctx, orc


def rel(a, b, floor=1e-300):
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def walker_rel(a, b):
    """Per walker, the largest element difference over the walker's largest element:
    max_pj |a_z,pj - b_z,pj| / max_pj |b_z,pj| for (W, M, N) stacks.  Every element is
    compared, so a wrong sign on a small element shows up (a norm ratio could hide it)."""
    W = a.shape[0]
    num = np.abs(a - b).reshape(W, -1).max(axis=1)
    return num / np.abs(b).reshape(W, -1).max(axis=1)


def assert_state_parity(ctx, orc, tol=1e-10):
    phi = ctx.get_walkers()
    assert walker_rel(phi, orc.phi).max() <= tol, walker_rel(phi, orc.phi).max()
    ov = ctx.get_overlaps()
    assert rel(ov, orc.ovlp).max() <= tol, rel(ov, orc.ovlp).max()
    w = ctx.get_weights()
    wref = orc.w.astype(np.complex128)
    scale = np.max(np.abs(wref))
    assert np.all(np.abs(w - wref) <= tol * np.maximum(np.abs(wref), 1e-3 * scale)), \
        np.max(np.abs(w - wref) / np.maximum(np.abs(wref), 1e-300))


def assert_energy_parity(ctx, orc, tol=1e-10):
    e, emix = ctx.local_energy()
    eref, emix_ref = orc.local_energy()
    for k in range(4):
        scale = np.maximum(np.abs(eref[:, k]), 1e-3 * np.abs(eref[:, 3]))
        assert np.all(np.abs(e[:, k] - eref[:, k]) <= tol * scale), (k, np.max(np.abs(e[:, k] - eref[:, k]) / scale))
    assert abs(emix - emix_ref) <= tol * abs(emix_ref)
    return e, emix
