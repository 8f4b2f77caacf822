"""GPU parity of the compact layout (arrays of the 3^r gasket cells only)
against the CPU oracle: pack and unpack bit-exact over every level up to 11,
every tile side and both walking orders; the write pass bit-exact for every
value kind and both element types; the CA step bit-exact and diffusion within
the FP64 tolerance, and both equal to the embedded GPU steps bit for bit.  At
the stencil workloads' full level the compact steps are checked against the
embedded ones (which the oracle checks on light-cone windows)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1706_04552_gb300 as sg  # noqa: E402
from paper_1706_04552_gb300 import inputs, workloads  # noqa: E402

from test_gpu_parity import DIFF_TOL, max_rel_err, rhos_for, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
ORDERS = ("rowmajor", "interleaved")


def dev1(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host1(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _s(rho):
    return rho.bit_length() - 1


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("r", [0, 1, 2, 3, 5, 6, 7, 9, 11])
def test_pack_unpack_match_oracle(orc, r, dtype, order):
    n = 1 << r
    rng = np.random.default_rng(40 + r)
    if dtype == "u8":
        grid = rng.integers(0, 256, (n, n), dtype=np.uint8)
        before = rng.integers(0, 256, (n, n), dtype=np.uint8)
    else:
        grid = rng.standard_normal((n, n)).astype(np.float32)
        before = rng.standard_normal((n, n)).astype(np.float32)
    oid = sg.ORDERS[order]
    g = to_dev(grid)
    for rho in rhos_for(r):
        s = _s(rho)
        c = torch.zeros(3 ** r, dtype=g.dtype, device=DEV)
        sg.compact_pack(g, c, r, rho, order=order)
        want = orc.compact_pack(r, s, grid, oid)
        assert np.array_equal(host1(c).view(np.uint8), want.view(np.uint8)), (rho, "pack")
        # unpack writes exactly the gasket cells
        b = to_dev(before)
        sg.compact_unpack(c, b, r, rho, order=order)
        want_b = orc.compact_unpack(r, s, want, before.copy(), oid)
        got_b = host1(b).reshape(n, n)
        assert np.array_equal(got_b.view(np.uint8), want_b.view(np.uint8)), (rho, "unpack")


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("r", [1, 4, 6, 8, 10])
def test_compact_write_matches_oracle(orc, r, dtype, order):
    n = 1 << r
    np_dt = np.uint8 if dtype == "u8" else np.float32
    oid = sg.ORDERS[order]
    for value, vid, vs in (("hash", orc.VAL_HASH, 7), ("linear31", orc.VAL_LINEAR31, 0),
                           ("const", orc.VAL_CONST, 0x40490FDB if dtype == "f32" else 201)):
        grid = np.zeros((n, n), dtype=np_dt)
        orc.map_write(r, grid, vid, vs)
        for rho in rhos_for(r):
            c = torch.full((3 ** r,), 3, dtype=torch.uint8 if dtype == "u8" else torch.float32,
                           device=DEV)
            sg.compact_map_write(c, r, rho, value, vs, order=order)
            want = orc.compact_pack(r, _s(rho), grid, oid)
            assert np.array_equal(host1(c).view(np.uint8), want.view(np.uint8)), (value, rho)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("r,p", [(0, 1.0), (1, 1.0), (2, 0.6), (4, 0.5), (6, 0.4), (8, 0.35),
                                 (10, 0.3)])
def test_compact_ca_matches_oracle(orc, r, p, order):
    oid = sg.ORDERS[order]
    s0 = inputs.ca_seed_grid(r, p, 11 + r)
    for rho in rhos_for(r):
        s = _s(rho)
        want = orc.compact_pack(r, s, s0, oid)
        a = dev1(want)
        b = torch.zeros_like(a)
        for step in range(5):
            sg.compact_ca_step(a, b, r, rho, order=order)
            want = orc.compact_ca_step(r, s, want, oid)
            assert np.array_equal(host1(b), want), (rho, step)
            a, b = b, a


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("r", [0, 1, 3, 5, 7, 9])
def test_compact_diffusion_matches_fp64_oracle(orc, r, order):
    oid = sg.ORDERS[order]
    u0 = inputs.uniform_grid(r, 21 + r)
    for rho in rhos_for(r):
        s = _s(rho)
        want = orc.compact_pack(r, s, u0, oid).astype(np.float64)
        a = dev1(orc.compact_pack(r, s, u0, oid))
        b = torch.zeros_like(a)
        for step in range(4):
            sg.compact_diffuse_step(a, b, r, rho, 0.2, order=order)
            want = orc.compact_diffuse_step(r, s, want, 0.2, oid)
            assert max_rel_err(host1(b), want) <= DIFF_TOL, (rho, step)
            a, b = b, a


@pytest.mark.parametrize("r", [6, 9, 11])
def test_compact_steps_equal_embedded_steps(r):
    # the same per-cell arithmetic: pack(embedded step) == compact step, bit for bit
    n = 1 << r
    s0 = to_dev(inputs.ca_seed_grid(r, 0.35, 5))
    u0 = to_dev(inputs.uniform_grid(r, 5))
    for rho in [p for p in (4, 16, 32, 64) if p <= n]:
        for order in ORDERS:
            emb = torch.zeros_like(s0)
            sg.ca_step(s0, emb, r, min(rho, 64), "lambda")
            ci = sg.compact_pack(s0, torch.empty(3 ** r, dtype=torch.uint8, device=DEV), r, rho,
                                 order=order)
            co = torch.empty_like(ci)
            sg.compact_ca_step(ci, co, r, rho, order=order)
            want = sg.compact_pack(emb, torch.empty_like(ci), r, rho, order=order)
            assert torch.equal(co, want), ("ca", rho, order)
            emb = torch.zeros_like(u0)
            sg.diffuse_step(u0, emb, r, rho, 0.2, "lambda")
            ci = sg.compact_pack(u0, torch.empty(3 ** r, dtype=torch.float32, device=DEV), r,
                                 rho, order=order)
            co = torch.empty_like(ci)
            sg.compact_diffuse_step(ci, co, r, rho, 0.2, order=order)
            want = sg.compact_pack(emb, torch.empty_like(ci), r, rho, order=order)
            assert torch.equal(co, want), ("diffusion", rho, order)


def test_compact_inputs_are_left_unchanged():
    r, rho = 8, 16
    a = dev1(np.random.default_rng(1).integers(0, 2, 3 ** r, dtype=np.uint8))
    keep = a.clone()
    sg.compact_ca_step(a, torch.empty_like(a), r, rho)
    u = dev1(np.random.default_rng(1).random(3 ** r).astype(np.float32))
    ukeep = u.clone()
    sg.compact_diffuse_step(u, torch.empty_like(u), r, rho)
    torch.cuda.synchronize()
    assert torch.equal(a, keep) and torch.equal(u, ukeep)


@pytest.mark.slow
def test_compact_full_size_matches_embedded():
    # the stencil workloads' level: 16 CA steps and 10 diffusion steps on the
    # compact arrays equal the embedded kernels' steps, packed; the write pass
    # at level 16 equals the embedded fill pass, packed
    w = workloads.STENCILS
    r = max(w["levels"])
    n = 1 << r
    rho = 64
    idx, vals = inputs.ca_seed_sparse(r, w["ca_p"], w["ca_seed"])
    a = torch.zeros(n * n, dtype=torch.uint8, device=DEV)
    a[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(vals).to(DEV)
    ca = sg.compact_pack(a, torch.empty(3 ** r, dtype=torch.uint8, device=DEV), r, rho)
    cb = torch.empty_like(ca)
    b = torch.zeros_like(a)
    for _ in range(16):
        sg.ca_step(a, b, r, w["ca_rho"], "lambda")
        a, b = b, a
        sg.compact_ca_step(ca, cb, r, rho)
        ca, cb = cb, ca
    assert torch.equal(ca, sg.compact_pack(a, torch.empty_like(ca), r, rho))
    del a, b, ca, cb
    idx, vals = inputs.uniform_sparse(r, w["diff_seed"])
    u = torch.zeros(n * n, dtype=torch.float32, device=DEV)
    u[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(vals).to(DEV)
    cu = sg.compact_pack(u, torch.empty(3 ** r, dtype=torch.float32, device=DEV), r, rho)
    cv = torch.empty_like(cu)
    v = torch.zeros_like(u)
    for _ in range(10):
        sg.diffuse_step(u, v, r, w["diff_rho"], w["alpha"], "lambda")
        u, v = v, u
        sg.compact_diffuse_step(cu, cv, r, rho, w["alpha"])
        cu, cv = cv, cu
    assert torch.equal(cu, sg.compact_pack(u, torch.empty_like(cu), r, rho))
    del u, v, cu, cv
    rw = workloads.WRITE_HEADLINE["r"]
    g = torch.zeros(1 << (2 * rw), dtype=torch.uint8, device=DEV)
    sg.map_write(g, rw, 64, "lambda_unroll", "hash", 1, store="fill")
    c = torch.empty(3 ** rw, dtype=torch.uint8, device=DEV)
    sg.compact_map_write(c, rw, 64, "hash", 1)
    assert torch.equal(c, sg.compact_pack(g, torch.empty_like(c), rw, 64))


FUSED_KS = (2, 3, 4, 5, 8, 9, 15, 16)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("r,p", [(6, 0.5), (7, 0.45), (8, 0.4), (10, 0.3)])
def test_compact_fused_ca_matches_oracle(orc, r, p, order):
    oid = sg.ORDERS[order]
    s0 = inputs.ca_seed_grid(r, p, 50 + r)
    ref = [orc.compact_pack(r, 6, s0, oid)]
    for _ in range(max(FUSED_KS)):
        ref.append(orc.compact_ca_step(r, 6, ref[-1], oid))
    a = dev1(ref[0])
    for k in FUSED_KS:
        b = torch.zeros_like(a)
        sg.compact_ca_steps(a, b, r, 64, k, order=order)
        assert np.array_equal(host1(b), ref[k]), k
    assert np.array_equal(host1(a), ref[0])             # the input is left as it was


def test_compact_fused_ca_equals_single_steps():
    r = 11
    s0 = sg.compact_pack(to_dev(inputs.ca_seed_grid(r, 0.35, 8)),
                         torch.empty(3 ** r, dtype=torch.uint8, device=DEV), r, 64)
    for k in (2, 7, 16):
        a, b = s0.clone(), torch.zeros_like(s0)
        for _ in range(k):
            sg.compact_ca_step(a, b, r, 64)
            a, b = b, a
        f = torch.zeros_like(s0)
        sg.compact_ca_steps(s0, f, r, 64, k)
        assert torch.equal(a, f), k


@pytest.mark.slow
def test_compact_fused_ca_full_size_matches_embedded_fused():
    # the stencil workload's CA sequence (256 steps from the seeded state) as
    # 16 launches of 16 fused compact steps equals the embedded fused run, packed
    w = workloads.STENCILS
    r = max(w["levels"])
    n = 1 << r
    idx, vals = inputs.ca_seed_sparse(r, w["ca_p"], w["ca_seed"])
    a = torch.zeros(n * n, dtype=torch.uint8, device=DEV)
    a[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(vals).to(DEV)
    ca = sg.compact_pack(a, torch.empty(3 ** r, dtype=torch.uint8, device=DEV), r, 64)
    cb = torch.empty_like(ca)
    b = torch.zeros_like(a)
    for _ in range(w["ca_steps"] // 16):
        sg.ca_steps(a, b, r, 64, 16)
        a, b = b, a
        sg.compact_ca_steps(ca, cb, r, 64, 16)
        ca, cb = cb, ca
    assert torch.equal(ca, sg.compact_pack(a, torch.empty_like(ca), r, 64))


@pytest.mark.slow
def test_compact_steps_at_the_largest_level():
    # level 16 (43 M cells; the embedded buffers are 4.3 GB u8 / 17.2 GB f32):
    # the compact CA (single and fused) and diffusion steps equal the packed
    # embedded steps bit for bit
    r, rho = 16, 64
    n = 1 << r
    idx, vals = inputs.ca_seed_sparse(r, 0.3, 5)
    a = torch.zeros(n * n, dtype=torch.uint8, device=DEV)
    a[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(vals).to(DEV)
    ca = sg.compact_pack(a, torch.empty(3 ** r, dtype=torch.uint8, device=DEV), r, rho)
    b = torch.zeros_like(a)
    sg.ca_steps(a, b, r, rho, 4)
    want = sg.compact_pack(b, torch.empty_like(ca), r, rho)
    got = torch.empty_like(ca)
    sg.compact_ca_steps(ca, got, r, rho, 4)
    assert torch.equal(got, want)
    c1, c2 = ca.clone(), torch.empty_like(ca)
    for _ in range(4):
        sg.compact_ca_step(c1, c2, r, rho)
        c1, c2 = c2, c1
    assert torch.equal(c1, want)
    del a, b, ca, want, got, c1, c2
    torch.cuda.empty_cache()
    idx, vals = inputs.uniform_sparse(r, 5)
    u = torch.zeros(n * n, dtype=torch.float32, device=DEV)
    u[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(vals).to(DEV)
    cu = sg.compact_pack(u, torch.empty(3 ** r, dtype=torch.float32, device=DEV), r, rho)
    v = torch.zeros_like(u)
    sg.diffuse_step(u, v, r, rho, 0.2, "lambda")
    want = sg.compact_pack(v, torch.empty_like(cu), r, rho)
    got = torch.empty_like(cu)
    sg.compact_diffuse_step(cu, got, r, rho, 0.2)
    assert torch.equal(got, want)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("r", [6, 9, 12])
def test_compact_write_into_pinned_host_memory(orc, r, dtype):
    np_dt = np.uint8 if dtype == "u8" else np.float32
    grid = np.zeros((1 << r, 1 << r), dtype=np_dt)
    orc.map_write(r, grid, orc.VAL_HASH, 4)
    for rho in (16, 64):
        h = torch.full((3 ** r,), 7, dtype=torch.uint8 if dtype == "u8" else torch.float32
                       ).pin_memory()
        sg.compact_map_write_mapped(h, r, rho, "hash", 4)
        torch.cuda.synchronize()
        want = orc.compact_pack(r, rho.bit_length() - 1, grid)
        assert np.array_equal(h.numpy().view(np.uint8), want.view(np.uint8)), rho
