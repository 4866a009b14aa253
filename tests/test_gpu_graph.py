"""CUDA-graph replay, batched uneven systems and the autotuner (GPU).

A replayed graph runs the same kernels in the same order as eager stepping, so its
walkers, weights and energies must be bit-identical; a batch of uneven systems in
one graph must reproduce each system stepped on its own, and in FP64 match the
oracle at 1e-10, with per-system branches and with grouped launches alike; autotuned tiles change only the order of floating-point sums
(results within 1e-12 relative in FP64, and the FP64 path still matches the oracle
at 1e-10).
"""
import numpy as np
import pytest

from gpu_common import assert_energy_parity, assert_state_parity, make_pair, need_gpu
from oracle import philox
from paper_2209_04015_b300.synthetic import make_c4, make_config, make_system, perturbed_walkers

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def new_ctx(s, W, phi=None, **kw):
    from paper_2209_04015_b300 import AfqContext
    ctx = AfqContext(dt=0.005, qr_period=5, **kw)
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    ctx.init_trial(s.psi_a, s.psi_b)
    ctx.init_walkers(W, phi)
    return ctx


def eager(ctx, nsteps):
    for _ in range(nsteps):
        ctx.propagate(None, 1)
        e, emix = ctx.local_energy()
    return e, emix


def same(a, b):
    assert np.array_equal(a.get_walkers(), b.get_walkers())
    assert np.array_equal(a.get_weights(), b.get_weights())
    assert np.array_equal(a.get_overlaps(), b.get_overlaps())


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_graph_replay_is_bit_identical_to_eager(precision):
    s = make_system(37, 5, 3, 71, seed=4, decay="geometric")
    phi = perturbed_walkers(s, 13, eps=0.3, seed=2)
    a = new_ctx(s, 13, phi, precision=precision)
    b = new_ctx(s, 13, phi, precision=precision)
    e_ref, emix_ref = eager(a, 10)
    b.graph_capture(5)
    b.graph_launch(2)
    e, emix = b.get_energy()
    assert b.get_step() == a.get_step() == 10
    same(a, b)
    assert np.array_equal(e, e_ref) and emix == emix_ref
    with pytest.raises(Exception):
        b.graph_capture(3)  # not a whole QR period


def test_batch_of_uneven_systems_matches_individual_contexts():
    from paper_2209_04015_b300 import AfqBatch
    shapes = [(20, 4, 3, 50, 16, "fp64"), (37, 5, 3, 71, 13, "fp64"), (48, 10, 10, 240, 24, "split_bf16"),
              (33, 2, 6, 40, 7, "split_bf16")]
    batch_ctx, solo_ctx = [], []
    for k, (M, na, nb, X, W, prec) in enumerate(shapes):
        s = make_system(M, na, nb, X, seed=10 + k, decay="geometric")
        phi = perturbed_walkers(s, W, eps=0.2, seed=k)
        batch_ctx.append(new_ctx(s, W, phi, precision=prec, seed=100 + k))
        solo_ctx.append(new_ctx(s, W, phi, precision=prec, seed=100 + k))
    b = AfqBatch(batch_ctx)
    b.capture(5)
    b.launch(3)
    b.synchronize()
    for bc, sc in zip(batch_ctx, solo_ctx):
        e_ref, _ = eager(sc, 15)
        e, _ = bc.get_energy()
        same(bc, sc)
        assert np.array_equal(e, e_ref)
    b.close()


def test_c4_batch_in_split_precision_matches_individual():
    """The eight uneven systems of the batched workload (48..220 orbitals, 0.2 M
    electrons per spin, X = 5 M, 512..32 walkers) in one graph, one QR period."""
    from paper_2209_04015_b300 import AfqBatch
    systems = make_c4()
    bctx = [new_ctx(s, W, precision="split_bf16", seed=7 + k) for k, (s, W) in enumerate(systems)]
    b = AfqBatch(bctx)
    b.capture(5)
    b.launch(1)
    b.synchronize()
    for k, (s, W) in enumerate(systems):
        ref = new_ctx(s, W, precision="split_bf16", seed=7 + k)
        e_ref, _ = eager(ref, 5)
        e, _ = bctx[k].get_energy()
        assert np.array_equal(e, e_ref)
        assert np.all(np.isfinite(e))
        ref.close()
    b.close()


@pytest.mark.parametrize("grouped", [False, True])
def test_c4_batch_in_fp64_matches_oracle(grouped):
    """The batched workload in FP64 (eight uneven systems: 48..220 orbitals, 0.2 M
    electrons per spin, X = 5 M, 512..32 walkers) stepped by one graph for one QR
    period with device Philox fields, against the oracle: two walkers of every system
    re-run by the oracle alone with the same counter-based field stream drawn by its
    own Philox (walkers are independent and the counters are keyed by walker index).
    Walkers, overlaps, weights and every energy part within 1e-10 relative.  grouped:
    the VHS build and the propagation of all eight systems as one persistent launch
    each per step."""
    from oracle.afqmc import Oracle
    from paper_2209_04015_b300 import AfqBatch
    systems = make_c4()
    nsteps = 5
    phis = [perturbed_walkers(s, W, eps=0.3, seed=30 + k) for k, (s, W) in enumerate(systems)]
    bctx = [new_ctx(s, W, phis[k], seed=7 + k) for k, (s, W) in enumerate(systems)]
    for c in bctx:
        c.autotune()
    b = AfqBatch(bctx, grouped=grouped)
    b.capture(nsteps)
    b.launch(1)
    b.synchronize()
    for k, (s, W) in enumerate(systems):
        ctx = bctx[k]
        idx = np.array([0, W - 1])
        orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, dt=0.005, qr_period=5)
        orc.init_walkers(phis[k][idx])
        orc.propagate([philox.gaussian_fields(t, W, s.X, 7 + k)[idx] for t in range(nsteps)])
        e, emix = ctx.get_energy()
        eref, _ = orc.local_energy()
        phi = ctx.get_walkers()[idx]
        dphi = (np.abs(phi - orc.phi).reshape(2, -1).max(axis=1) /
                np.abs(orc.phi).reshape(2, -1).max(axis=1))
        assert dphi.max() <= 1e-10, (k, dphi)
        assert np.max(np.abs(ctx.get_overlaps()[idx] - orc.ovlp) / np.abs(orc.ovlp)) <= 1e-10
        w = ctx.get_weights()[idx].real
        assert np.all(np.abs(w - orc.w) <= 1e-10 * np.abs(orc.w)), (k, w, orc.w)
        for part in range(4):
            scale = np.maximum(np.abs(eref[:, part]), 1e-3 * np.abs(eref[:, 3]))
            assert np.all(np.abs(e[idx, part] - eref[:, part]) <= 1e-10 * scale), (k, part)
    b.close()
    for c in bctx:
        c.close()


@pytest.mark.parametrize("workload", ["uneven", "c4"])
def test_grouped_batch_is_bit_identical_to_per_system_launches(workload):
    """Grouped launches (one persistent VHS build and one persistent propagation over
    every system's tiles per step, tiles from a per-system descriptor table) against
    the per-system graph branches, two QR periods: the same kernels' arithmetic per
    tile, so walkers, weights, overlaps and energies are bit-identical.  The uneven set
    has ragged column chunks, several units per CTA and a system with one walker;
    the c4 set is the batched workload, autotuned (its per-system column chunks differ
    from the grouped launch's)."""
    from paper_2209_04015_b300 import AfqBatch
    if workload == "uneven":
        shapes = [(20, 4, 3, 50, 16), (37, 5, 3, 71, 13), (9, 2, 1, 12, 1), (64, 7, 7, 120, 5),
                  (33, 2, 6, 40, 7)]
        systems = [(make_system(M, na, nb, X, seed=40 + k, decay="geometric"), W)
                   for k, (M, na, nb, X, W) in enumerate(shapes)]
    else:
        systems = make_c4()
    phis = [perturbed_walkers(s, W, eps=0.3, seed=50 + k) for k, (s, W) in enumerate(systems)]
    sets = []
    for grouped in (False, True):
        ctxs = [new_ctx(s, W, phis[k], seed=3 + k) for k, (s, W) in enumerate(systems)]
        if workload == "c4":
            for c in ctxs:
                c.autotune()
        b = AfqBatch(ctxs, grouped=grouped)
        b.capture(5)
        b.launch(2)
        b.synchronize()
        sets.append((b, ctxs))
    (b0, per_system), (b1, grouped_ctxs) = sets
    for a, g in zip(per_system, grouped_ctxs):
        same(a, g)
        ea, ma = a.get_energy()
        eg, mg = g.get_energy()
        assert np.array_equal(ea, eg) and ma == mg
        assert a.get_step() == g.get_step() == 10
    for b, ctxs in sets:
        b.close()
        for c in ctxs:
            c.close()


def test_grouped_batch_takes_fp64_contexts_only():
    from paper_2209_04015_b300 import AfqBatch
    from paper_2209_04015_b300.afqmc import AFQ_ERR_ARG, AfqError
    s = make_system(37, 5, 3, 71, seed=4, decay="geometric")
    ctxs = [new_ctx(s, 4), new_ctx(s, 4, precision="split_bf16")]
    with pytest.raises(AfqError) as e:
        AfqBatch(ctxs, grouped=True)
    assert e.value.code == AFQ_ERR_ARG
    for c in ctxs:
        c.close()


def test_autotune_fp64_keeps_parity():
    s = make_system(37, 5, 3, 71, seed=4, decay="geometric", e0=0.37)
    W = 13
    phi = perturbed_walkers(s, W, eps=0.3, seed=2)
    ctx, orc = make_pair(s, W, phi=phi)
    e0, _ = ctx.local_energy()
    ctx.autotune()
    tiles = ctx.get_tiles()
    assert tiles[0] >= 1 and tiles[1] in (2, 4, 8)
    e1, _ = ctx.local_energy()
    assert np.max(np.abs(e1 - e0) / np.abs(e0[:, 3:4])) < 1e-12
    fields = np.stack([philox.gaussian_fields(k, W, s.X, 1) for k in range(6)])
    ctx.propagate(fields, 6)
    orc.propagate(list(fields))
    assert_state_parity(ctx, orc, 1e-10)
    assert_energy_parity(ctx, orc, 1e-10)


@pytest.mark.parametrize("exchange", ["direct", "stored"])
def test_autotune_split_keeps_energies(exchange):
    s, c = make_config("c2")
    W = c["W"]
    phi = perturbed_walkers(s, W, eps=0.3, seed=2)
    ctx = new_ctx(s, W, phi, precision="split_bf16", exchange=exchange)
    e0, _ = ctx.local_energy()
    ctx.autotune()
    tiles = ctx.get_tiles()
    assert tiles[4] >= 1                       # force-bias split-K depth
    if exchange == "direct":                   # walkers per direct exchange tile
        assert tiles[2] >= 1 and tiles[3] >= 1
    e1, _ = ctx.local_energy()
    assert np.max(np.abs(e1[:, 3] - e0[:, 3])) < 1e-6
