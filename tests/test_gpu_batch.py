"""GPU checks of the batched Sigma entry points (gf2_batch_*, gf2_sigma_tau_batched).

A batch of systems of uneven size (N = 4 .. 64, among them N = 36, 40 and 50)
runs through the autotuner and one recorded CUDA graph, with BF16 pairs of
instances sharing one block-diagonal 64-wide system; every instance's
Sigma(tau) is compared with the oracle's Eq. Sigma
at the tolerance of the path the tuner chose (FP64: 1e-10 relative; FP16x3 and
BF16x6 split: 3e-6 relative, as in the single-system split tests).  A second
call replays the graph on new contents of the same buffers.
"""

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import sigma as osg

pytestmark = pytest.mark.gpu

# (N, n_tau), uneven on purpose; with a BF16 split the tuner pairs two of the
# N = 36, 40, 50 instances with the smaller ones of the same grid (24, 12) into
# block-diagonal 64-wide systems; N = 64 finds no partner
SIZES = [(4, 33), (10, 33), (17, 33), (40, 17), (64, 17), (36, 17), (24, 17), (50, 17), (12, 17)]
TOL = {0: 1e-10, 2: 3e-6, 3: 3e-6}


@pytest.fixture(scope="module")
def g():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import os
    import paper_1405_3273_gb300 as g
    from paper_1405_3273_gb300 import build
    if not os.path.exists(g.LIB_PATH):
        build.build()
    g.lib()
    return g


@pytest.fixture(scope="module")
def systems():
    out = []
    for idx, (n, n_tau) in enumerate(SIZES):
        G = gi.random_symmetric_g(n, n_tau, seed=300 + idx)
        v = gi.random_eri(n, seed=400 + idx)
        out.append((G, v, osg.sigma_tau(G, v)))
    return out


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("prec", [3, 2])
def test_batched_sigma_matches_oracle_and_replays(g, systems, prec):
    b = g.Batch([n for n, _ in SIZES], [t for _, t in SIZES])
    try:
        Gs = [dev(G) for G, _, _ in systems]
        outs = [torch.zeros_like(x) for x in Gs]
        for i, (_, v, _) in enumerate(systems):
            g.gf2_batch_set_system(b.handle, i, dev(v))
        g.gf2_sigma_tau_batched(b.handle, Gs, outs, prec)
        plans = [g.gf2_batch_plan(b.handle, i) for i in range(len(SIZES))]
        print("plan (path, est ms, lane, slots per launch):", plans)
        assert all(p[3] in (16, 32) for p in plans)
        assert all(p[0] in (0, prec) for p in plans)
        assert plans[4][0] == prec, "N = 64 should take the tensor-core path"
        partners = [g.gf2_batch_partner(b.handle, i) for i in range(len(SIZES))]
        print("partners:", partners)
        for i, q in enumerate(partners):
            if q >= 0:
                assert partners[q] == i and SIZES[i][0] + SIZES[q][0] <= 64 and SIZES[i][1] == SIZES[q][1]
        if prec == 2:  # BF16: the 33..50 instances share their tiles where a partner fits
            # two smaller instances on the 17-point grid (24, 12) for three larger ones
            assert sum(q >= 0 for q in partners) == 4 and partners[4] == -1
            assert all(plans[i][1] == 0.0 for i, q in enumerate(partners) if q >= 0 and SIZES[i][0] < SIZES[q][0])
        else:          # FP16 scales are per time point: never shared
            assert all(q == -1 for q in partners)
        # (for N = 4 the two paths take about the same time; either choice is valid)
        for i, (_, _, ref) in enumerate(systems):
            rel = np.abs(outs[i].cpu().numpy() - ref).max() / np.abs(ref).max()
            print(f"instance {i} N={SIZES[i][0]} path {plans[i][0]}: max rel err {rel:.2e}")
            assert rel <= TOL[plans[i][0]], i
        # replay on new contents of the same buffers: G -> G/2 scales Sigma by 1/8
        for x in Gs:
            x.mul_(0.5)
        for x in outs:
            x.fill_(float("nan"))
        g.gf2_sigma_tau_batched(b.handle, Gs, outs, prec)
        for i, (_, _, ref) in enumerate(systems):
            rel = np.abs(outs[i].cpu().numpy() - ref / 8).max() / np.abs(ref / 8).max()
            assert rel <= TOL[plans[i][0]], i
    finally:
        b.close()


def test_batched_sigma_equals_single_system_calls(g, systems):
    """The batch runs the same kernels as gf2_sigma_tau with the tuner's path."""
    b = g.Batch([n for n, _ in SIZES], [t for _, t in SIZES])
    try:
        Gs = [dev(G) for G, _, _ in systems]
        outs = [torch.zeros_like(x) for x in Gs]
        for i, (_, v, _) in enumerate(systems):
            g.gf2_batch_set_system(b.handle, i, dev(v))
        g.gf2_sigma_tau_batched(b.handle, Gs, outs, 3)
        for i, ((n, n_tau), (G, v, _)) in enumerate(zip(SIZES, systems)):
            path = g.gf2_batch_plan(b.handle, i)[0]
            with g.Context(n, n_tau, 8, 1.0) as ctx:
                g.gf2_set_integrals(ctx.handle, dev(v))
                one = torch.zeros_like(Gs[i])
                g.gf2_sigma_tau(ctx.handle, Gs[i], one, path)
                torch.cuda.synchronize()
            diff = (one - outs[i]).abs().max().item() / one.abs().max().item()
            assert diff <= 1e-12, (i, diff)
    finally:
        b.close()


def test_batched_rejects_null_buffers(g, systems):
    b = g.Batch([4, 10], [33, 33])
    try:
        import ctypes
        L = g.lib()
        st = L.gf2_sigma_tau_batched(b.handle, None, None, 3)
        assert st == 1
        assert "NULL" in g.gf2_batch_last_error(b.handle)
        with pytest.raises(g.GF2Error):
            g.gf2_batch_tune(b.handle, [dev(systems[0][0]), dev(systems[1][0])], 3)  # no integrals yet
        assert ctypes is not None
    finally:
        b.close()


def test_batched_fp64_every_instance_on_the_fp64_path(g, systems):
    """prec = FP64: the tuner has one admissible path; every instance within 1e-10 of the oracle."""
    sizes = SIZES[:4]
    b = g.Batch([n for n, _ in sizes], [t for _, t in sizes])
    try:
        Gs = [dev(G) for G, _, _ in systems[:4]]
        outs = [torch.zeros_like(x) for x in Gs]
        for i, (_, v, _) in enumerate(systems[:4]):
            g.gf2_batch_set_system(b.handle, i, dev(v))
        g.gf2_sigma_tau_batched(b.handle, Gs, outs, 0)
        for i, (_, _, ref) in enumerate(systems[:4]):
            assert g.gf2_batch_plan(b.handle, i)[0] == 0
            rel = np.abs(outs[i].cpu().numpy() - ref).max() / np.abs(ref).max()
            assert rel <= 1e-10, (i, rel)
    finally:
        b.close()


def test_batch_rejects_bad_instances_and_precisions(g, systems):
    b = g.Batch([4], [33])
    try:
        v = dev(systems[0][1])
        with pytest.raises(g.GF2Error):
            g.gf2_batch_set_system(b.handle, 1, v)          # instance out of range
        g.gf2_batch_set_system(b.handle, 0, v)
        with pytest.raises(g.GF2Error):
            g.gf2_batch_tune(b.handle, [dev(systems[0][0])], 9)   # unknown precision
        with pytest.raises(g.GF2Error):
            g.gf2_batch_plan(b.handle, 0)                   # not tuned yet
    finally:
        b.close()


def test_shared_tiles_with_overlaps_match_oracle(g):
    """Two chains with their overlaps (STO-3G H36 and H20 at 1.7 bohr, so the
    split path works in the orthonormal basis): the BF16x6 tuner pairs them
    into one block-diagonal system with a block-diagonal S; each instance's
    Sigma(tau) in the AO basis against the oracle's Eq. Sigma."""
    sizes, n_tau = [36, 20], 17
    b = g.Batch(sizes, [n_tau] * 2)
    try:
        Gs, outs, refs = [], [], []
        for i, n in enumerate(sizes):
            s = gi.build_system("chain", coords=gi.h_chain(n, 1.7), basis="sto-3g", beta=10.0, n_tau=n_tau, n_iw=8)
            G = gi.random_symmetric_g(n, n_tau, seed=700 + i) * 0.3
            refs.append(osg.sigma_tau(G, s.eri))
            g.gf2_batch_set_system(b.handle, i, dev(s.eri), dev(s.S))
            Gs.append(dev(G))
            outs.append(torch.zeros_like(Gs[-1]))
        g.gf2_sigma_tau_batched(b.handle, Gs, outs, 2)
        assert g.gf2_batch_partner(b.handle, 0) == 1 and g.gf2_batch_partner(b.handle, 1) == 0
        for i, ref in enumerate(refs):
            rel = np.abs(outs[i].cpu().numpy() - ref).max() / np.abs(ref).max()
            print(f"paired instance {i} N={sizes[i]} with S: max rel err {rel:.2e}")
            assert rel <= TOL[2], i
    finally:
        b.close()
