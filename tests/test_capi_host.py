"""C-ABI host checks (no GPU): the library loads and exports the header's
symbols, argument errors come back as status codes, and the host-side period
construction (gates, kick folding, fusion) agrees with the oracle."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2111_08044_gb300 import capi, inputs
from tests import dense_reference as dr


def test_library_exports_every_header_symbol(svlib):
    names = capi.header_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(svlib, n), n
    assert svlib.sv_version() >= 1


def test_create_without_device_is_an_error_code(svlib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = ctypes.c_void_p()
    rc = svlib.sv_create(ctypes.byref(ctx), 0, capi.SV_C64, None)
    assert rc == capi.SV_ECUDA
    assert not ctx.value


def test_argument_errors(svlib):
    p, _ = capi.make_params()
    out = np.zeros(64)
    assert svlib.sv_host_bond_gates(1, ctypes.byref(p), out.ctypes.data_as(capi._dp), None) == capi.SV_EINVAL
    assert svlib.sv_host_bond_gates(35, ctypes.byref(p), None, None) == capi.SV_EINVAL
    bad, _ = capi.make_params(K=0)
    assert svlib.sv_host_bond_gates(6, ctypes.byref(bad), None, None) == capi.SV_EINVAL
    bad, _ = capi.make_params(first_layer=2)
    assert svlib.sv_host_bond_gates(6, ctypes.byref(bad), None, None) == capi.SV_EINVAL
    bad, _ = capi.make_params(hx=float("nan"))
    assert svlib.sv_host_bond_gates(6, ctypes.byref(bad), None, None) == capi.SV_EINVAL
    n = ctypes.c_int(0)
    assert svlib.sv_host_fusion_plan(6, ctypes.byref(p), 8, ctypes.byref(n), None, None, None) == capi.SV_EINVAL
    assert svlib.sv_host_fusion_plan(6, ctypes.byref(p), 1, ctypes.byref(n), None, None, None) == capi.SV_EINVAL
    assert svlib.sv_host_period_gates(6, None, ctypes.byref(n), None, None) == capi.SV_EINVAL
    # a null context is rejected everywhere
    assert svlib.sv_init(None, 8, None) == capi.SV_EINVAL
    assert svlib.sv_evolve(None, 1, None, None) == capi.SV_EINVAL
    assert svlib.sv_expect_energy(None, None, None) == capi.SV_EINVAL
    assert svlib.sv_period_counter(None) == -1


def _lib_gates(svlib, L, **kw):
    p, keep = capi.make_params(**kw)
    g = np.zeros((L - 1, 4, 4), dtype=np.complex128)
    k = np.zeros((2, 2), dtype=np.complex128)
    assert svlib.sv_host_bond_gates(L, ctypes.byref(p), g.ctypes.data_as(capi._dp),
                                    k.ctypes.data_as(capi._dp)) == 0
    return g, k


@pytest.mark.parametrize("L,ew", [(2, 0.5), (5, 1.0), (12, 0.5)])
def test_bond_gates_match_oracle(svlib, L, ew):
    kw = dict(J=1.1, hx=0.8, hz=0.35, T=0.7, K=3, theta=0.41, edge_field_weight=ew)
    g, k = _lib_gates(svlib, L, **kw)
    hb = orc.ising_bond_hamiltonians(L, 1.1, 0.8, 0.35, ew)
    np.testing.assert_allclose(g, orc.bond_gates(hb, 0.7 / 3), atol=1e-13, rtol=0)
    np.testing.assert_allclose(k, orc.kick_gates(1, 0.41)[0], atol=1e-15, rtol=0)


def _period_gates(svlib, L, **kw):
    p, keep = capi.make_params(**kw)
    n = ctypes.c_int(0)
    assert svlib.sv_host_period_gates(L, ctypes.byref(p), ctypes.byref(n), None, None) == 0
    bonds = np.zeros(n.value, dtype=np.int32)
    mats = np.zeros((n.value, 4, 4), dtype=np.complex128)
    assert svlib.sv_host_period_gates(L, ctypes.byref(p), ctypes.byref(n),
                                      bonds.ctypes.data_as(capi._ip),
                                      mats.ctypes.data_as(capi._dp)) == 0
    return bonds, mats


@pytest.mark.parametrize("L,first", [(2, 0), (5, 0), (6, 1), (7, 1)])
def test_folded_period_equals_oracle_period(svlib, L, first):
    """Kick folding: the library's folded gate sequence multiplies out to the
    same Floquet operator as the oracle's unfolded one."""
    kw = dict(J=0.9, hx=1.1, hz=0.3, T=0.6, K=3, theta=0.27, first_layer=first)
    bonds, mats = _period_gates(svlib, L, **kw)
    assert len(bonds) == 3 * (L - 1)
    U = np.eye(1 << L, dtype=np.complex128)
    for b, m in zip(bonds, mats):
        U = dr.two_site_op(L, int(b), m) @ U
    hb = orc.ising_bond_hamiltonians(L, 0.9, 1.1, 0.3, 0.5)
    Ud = dr.floquet_dense([dr.ising_bond_dense(L, b, 0.9, 1.1, 0.3, 0.5) for b in range(L - 1)],
                          L, 0.2, 0.27, 3, first)
    np.testing.assert_allclose(U, Ud, atol=1e-12, rtol=0)
    # and against the oracle applying the same period to a random state
    sp = inputs.random_product_spinors(L, 3)
    psi = orc.product_state(sp)
    orc.period(psi, orc.bond_gates(hb, 0.2), orc.kick_gates(L, 0.27), 3, first)
    np.testing.assert_allclose(U @ orc.product_state(sp), psi, atol=1e-12, rtol=0)


def _plan(svlib, L, n, want_unitaries=False, **kw):
    p, keep = capi.make_params(**kw)
    cnt = ctypes.c_int(0)
    assert svlib.sv_host_fusion_plan(L, ctypes.byref(p), n, ctypes.byref(cnt), None, None,
                                     None) == 0
    P = cnt.value
    lo = np.zeros(P, dtype=np.int32)
    gc = np.zeros(P, dtype=np.int32)
    dim = 1 << n
    U = np.zeros((P, dim, dim), dtype=np.complex128) if L <= 12 or want_unitaries else None
    assert svlib.sv_host_fusion_plan(
        L, ctypes.byref(p), n, ctypes.byref(cnt), lo.ctypes.data_as(capi._ip),
        gc.ctypes.data_as(capi._ip), None if U is None else U.ctypes.data_as(capi._dp)) == 0
    return lo, gc, U


def _window_op(L, lo, n, U):
    """Embed an n-site unitary acting on sites lo..lo+n-1 (local bit j = site lo+j)."""
    return np.kron(np.kron(np.eye(1 << (L - lo - n)), U), np.eye(1 << lo))


@pytest.mark.parametrize("L,n", [(6, 3), (8, 4), (9, 5), (10, 6), (10, 7)])
def test_fused_passes_multiply_to_the_period(svlib, L, n):
    kw = dict(J=1.0, hx=0.9, hz=0.4, T=0.5, K=4, theta=0.3)
    lo, gc, U = _plan(svlib, L, n, **kw)
    assert gc.sum() == 4 * (L - 1)
    # a period may start at any window s <= 7: the state stays in that
    # window's layout between periods; the passes still compose to U_F
    assert 0 <= lo[0] <= 7
    total = np.eye(1 << L, dtype=np.complex128)
    for k in range(len(lo)):
        total = _window_op(L, lo[k], n, U[k]) @ total
    Ud = dr.floquet_dense([dr.ising_bond_dense(L, b, 1.0, 0.9, 0.4, 0.5) for b in range(L - 1)],
                          L, 0.125, 0.3, 4, 0)
    np.testing.assert_allclose(total, Ud, atol=1e-12, rtol=0)


def _nearest_digits(x):
    """The tensor-core digit value 2^-7 (u0 + u1/256 + u2/65536) with every
    digit an integer rounded to nearest (the scheme before the descent)."""
    y, out, sc = x * 128.0, np.zeros_like(x), 1.0 / 128.0
    for _ in range(3):
        d = np.rint(y)
        out, y, sc = out + d * sc, (y - d) * 256.0, sc / 256.0
    return out


def _defect(M):
    D = M.conj().T @ M - np.eye(M.shape[0])
    return D, float(np.sum(np.abs(D) ** 2) + np.trace(D).real ** 2)


@pytest.mark.parametrize("L", [14, 26])
def test_pass_operands_are_close_to_unitary(svlib, L):
    """Every block pass applies the same rounded copy of its fused unitary
    each period, so a defect Ur^H Ur - I changes the norm by the same amount
    every period.  The operands stay within the format's spacing of the FP64
    unitary, their defect is no larger than nearest rounding's, and the trace
    of the defect summed over the period's passes (the norm change per period
    of a maximally mixed state) is far below nearest rounding's."""
    n = 6
    p, _ = capi.make_params(mode=capi.SV_MODE_BLOCK, block_n=n)
    lo, gc, U = _plan(svlib, L, n, want_unitaries=True)
    trace_sum = {capi.SV_SPLIT_BF16X3: 0.0, capi.SV_SPLIT_FP32: 0.0}
    trace_near = dict(trace_sum)
    for k in range(len(lo)):
        for split in trace_sum:
            o = np.zeros(2 * 4 ** n)
            assert svlib.sv_host_pass_operand(L, ctypes.byref(p), n, k, split,
                                              o.ctypes.data_as(capi._dp)) == 0
            Ur = o.view(np.complex128).reshape(1 << n, 1 << n)
            err = np.maximum(np.abs((Ur - U[k]).real), np.abs((Ur - U[k]).imag))
            if split == capi.SV_SPLIT_BF16X3:
                # u0 integer; u1, u2 8-bit significands; the chosen u2 is one
                # of the two neighbours of its exact value: within 2^-25
                assert err.max() <= 2.0 ** -25
                Un = _nearest_digits(U[k].real) + 1j * _nearest_digits(U[k].imag)
                # the digits are exact bf16 values: u0/128 a multiple of 2^-7
                u0 = np.rint(U[k].real * 128.0)
                assert np.all(np.abs(u0) <= 128)
            else:
                spacing = np.spacing(np.abs(U[k].astype(np.complex64).real).astype(np.float32))
                assert np.all(np.abs((Ur - U[k]).real) <= spacing.astype(np.float64) * 1.0001)
                # each row's largest entry is applied with its residual (exact
                # to ~2^-48); every other entry is an FP32 value
                lead = np.argmax(np.abs(U[k]), axis=1)
                rows = np.arange(1 << n)
                assert np.all(np.abs(Ur[rows, lead] - U[k][rows, lead]) < 1e-13)
                rest = np.ones(Ur.shape, bool)
                rest[rows, lead] = False
                assert np.all(Ur.real[rest] == Ur.real[rest].astype(np.float32))
                assert np.all(Ur.imag[rest] == Ur.imag[rest].astype(np.float32))
                Un = U[k].astype(np.complex64).astype(np.complex128)
            D, f = _defect(Ur)
            Dn, fn = _defect(Un)
            assert f <= fn * 1.000001
            trace_sum[split] += np.trace(D).real / (1 << n)
            trace_near[split] += np.trace(Dn).real / (1 << n)
            if split == capi.SV_SPLIT_BF16X3:
                # the 8-bit last digits leave a much smaller defect
                assert np.linalg.norm(D) < 0.2 * np.linalg.norm(Dn)
    for split in trace_sum:
        assert abs(trace_sum[split]) < 2e-9, (split, trace_sum[split], trace_near[split])
        assert abs(trace_sum[split]) < 0.1 * abs(trace_near[split])


@pytest.mark.parametrize("L", [13, 20, 26, 30, 34])
@pytest.mark.parametrize("n", [6, 7])
def test_fusion_plan_shape_large_chains(svlib, L, n):
    lo, gc, _ = _plan(svlib, L, n)
    assert gc.sum() == 4 * (L - 1)
    assert 0 <= lo[0] <= 7  # one relabel pass reaches the start from site 0
    jumps = np.abs(np.diff(np.concatenate([lo, lo[:1]])))
    assert jumps.max() <= 7  # every relabel fits in a 7-bit row index
    assert len(lo) <= {6: 21, 7: 18}[n]


def test_batch_host_checks(svlib):
    import ctypes
    L = np.array([14, 22, 2], dtype=np.int32)
    total = svlib.sv_batch_state_bytes(3, L.ctypes.data_as(capi._ip))
    # 256-byte aligned chain slices of 8 * 2^L bytes
    assert total == (8 << 14) + (8 << 22) + (8 << 2)
    bad = np.array([14, 35], dtype=np.int32)
    assert svlib.sv_batch_state_bytes(2, bad.ctypes.data_as(capi._ip)) == 0
    b = ctypes.c_void_p()
    p = (capi.sv_floquet_params * 1)()
    assert svlib.sv_batch_create(ctypes.byref(b), 0, 0, None, p, None, None, 0, -1,
                                 None) == capi.SV_EINVAL
    assert not b.value


def _block_layout(svlib, L, n):
    p, _ = capi.make_params()
    cnt = ctypes.c_int(64)
    lo = (ctypes.c_int * 64)()
    assert svlib.sv_host_fusion_plan(L, ctypes.byref(p), n, ctypes.byref(cnt), lo, None, None) == 0
    P = cnt.value
    a = np.zeros(64, np.int32)
    sig = np.zeros(64 * 13, np.int32)
    rows = np.zeros(64 * 7, np.uint8)
    wf = np.zeros(64, np.int32)
    xs = np.zeros(64, np.int32)
    st = np.zeros(64 * 13, np.uint8)
    c2 = ctypes.c_int(64)
    assert svlib.sv_host_block_layout(L, ctypes.byref(p), n, ctypes.byref(c2),
                                      a.ctypes.data_as(capi._ip), sig.ctypes.data_as(capi._ip),
                                      rows.ctypes.data, wf.ctypes.data_as(capi._ip),
                                      xs.ctypes.data_as(capi._ip), st.ctypes.data) == 0
    assert c2.value == P
    los = [lo[k] for k in range(P)]
    # every site's <X> is measured exactly once per period
    measured = [los[k] + j for k in range(P) for j in range(n) if (xs[k] >> j) & 1]
    assert sorted(measured) == list(range(L))
    return (los, a[:P], sig[:13 * P].reshape(P, 13), rows[:7 * P].reshape(P, 7), wf[:P],
            st[:13 * P].reshape(P, 13))


def _site_position(L, n, lo, s):
    # window sites on the lowest n bits, sites below it next, the rest in place
    if lo <= s < lo + n:
        return s - lo
    return n + s if s < lo else s


@pytest.mark.parametrize("L", [13, 16, 20, 23, 26, 30, 34])
def test_block_tile_layout_and_row_map(svlib, L):
    """Each pass's relabel sigma follows the window layout rule; the
    tensor-core row map is invertible, keeps the converter's swizzled row
    reads conflict-free, and its reported staging wavefronts equal a
    brute-force bank count (rows and staging order as chosen) that never
    exceeds the natural order's; the staging order is a permutation that
    keeps bits 0-3 and leaves conflict-free passes in the natural order."""
    n, R = 6, min(7, L - 6)
    los, a, sig, rows, wf, st = _block_layout(svlib, L, n)
    P = len(los)
    for k in range(P):
        lo, lo_next = los[k], los[(k + 1) % P]
        tile_pos = list(range(n)) + [a[k] + b for b in range(R)]
        site_of = {_site_position(L, n, lo, s): s for s in range(L)}
        for q, pos in enumerate(tile_pos):
            out_pos = _site_position(L, n, lo_next, site_of[pos])
            want = out_pos if out_pos < n else tile_pos.index(out_pos)
            assert sig[k, q] == want, (k, q)
        if R < 7:
            assert wf[k] == 0 and not rows[k].any() and not st[k].any()
            continue
        assert sorted(st[k]) == list(range(13)) and list(st[k, :4]) == [0, 1, 2, 3]
        natural = list(st[k]) == list(range(13))
        rmap = [0] * 128
        for m in range(128):
            for i in range(7):
                if (m >> i) & 1:
                    rmap[m] ^= int(rows[k, i])
        assert sorted(rmap) == list(range(128))
        # converter: the 8 lanes of each quarter-warp read 8 different 16-byte chunks
        for m0 in range(0, 128, 8):
            assert len({rmap[m] & 7 for m in range(m0, m0 + 8)}) == 8

        def wavefronts(rowmap, spos):
            # a 64-bit shared store is served per half-warp: each half takes
            # as many wavefronts as the most lanes on one 8-byte bank slot
            worst = 0
            for q in range(4):
                for c in (0, 21, 63):
                    total = 0
                    for half in range(2):
                        slots = {}
                        for t in range(16 * half, 16 * half + 16):
                            y = c | (rowmap[32 * q + t] << n)
                            yo = sum(((y >> b) & 1) << int(spos[sig[k, b]]) for b in range(13))
                            byte = 8 * yo
                            byte ^= ((byte >> 7) & 7) << 4
                            slots.setdefault((byte >> 3) & 15, set()).add(byte)
                        total += max(len(v) for v in slots.values())
                    worst = max(worst, total)
            return worst
        got = wavefronts(rmap, st[k])
        assert got == wf[k], (k, got, wf[k])
        assert got <= wavefronts(list(range(128)), list(range(13)))
        assert natural or got < 16
    if L == 30:
        # the row map spreads every relabelled write of the L = 30 period
        # (16 passes from the start at site 2) to at most 4 wavefronts
        assert max(wf) <= 4
    if L in (16, 23):
        # one pass sends six row bits above the bank bits: no row map helps
        # (16 wavefronts), a reordered staging tile does
        k = {16: 6, 23: 11}[L]
        assert list(st[k]) != list(range(13)) and wf[k] <= 4


@pytest.mark.parametrize("L,first", [(6, 0), (7, 1)])
def test_inverse_period_is_the_adjoint(svlib, L, first):
    """inverse = 1 gives the forward folded gates in reverse order, each
    replaced by its adjoint, so that one inverse period undoes U_F (the echo
    of Sec. V), against the dense Floquet operator."""
    kw = dict(J=0.9, hx=1.1, hz=0.3, T=0.6, K=3, theta=0.27, first_layer=first)
    bonds, mats = _period_gates(svlib, L, **kw)
    ibonds, imats = _period_gates(svlib, L, inverse=1, **kw)
    np.testing.assert_array_equal(ibonds, bonds[::-1])
    for k in range(len(bonds)):
        np.testing.assert_allclose(imats[k], mats[-1 - k].conj().T, atol=0, rtol=0)
    Ui = np.eye(1 << L, dtype=np.complex128)
    for b, m in zip(ibonds, imats):
        Ui = dr.two_site_op(L, int(b), m) @ Ui
    Ud = dr.floquet_dense([dr.ising_bond_dense(L, b, 0.9, 1.1, 0.3, 0.5) for b in range(L - 1)],
                          L, 0.2, 0.27, 3, first)
    np.testing.assert_allclose(Ui, Ud.conj().T, atol=1e-12, rtol=0)


def test_inverse_flag_checks(svlib):
    n = ctypes.c_int(0)
    p, _ = capi.make_params(inverse=2)
    assert svlib.sv_host_period_gates(6, ctypes.byref(p), ctypes.byref(n), None, None) == capi.SV_EINVAL
    p, _ = capi.make_params(inverse=1, theta_p=[0.1, 0.2])
    assert svlib.sv_host_period_gates(6, ctypes.byref(p), ctypes.byref(n), None, None) == capi.SV_EINVAL


def _store_view(svlib, L, p, k):
    rank = ctypes.c_int(0)
    dims = (ctypes.c_ulonglong * 5)()
    strides = (ctypes.c_ulonglong * 4)()
    box = (ctypes.c_uint * 5)()
    coord = (ctypes.c_int * 4)()
    assert svlib.sv_host_store_view(L, ctypes.byref(p), 6, k, ctypes.byref(rank), dims, strides,
                                    box, coord) == 0
    r = rank.value
    return r, list(dims)[:r], [8] + list(strides)[:r - 1], list(box)[:r], list(coord)


@pytest.mark.parametrize("L,first", [(13, 0), (14, 0), (16, 0), (19, 0), (21, 0), (21, 1), (23, 0),
                                     (27, 0), (30, 0)])
def test_tensor_core_store_view_places_every_amplitude(svlib, L, first):
    """The TMA store view of every tensor-core pass, walked on the host: the
    staging element that holds output amplitude y of tile t (staging bit
    spos[o] = output bit o) lands on the state index the pass writes, i.e.
    output bits 0-5 on state bits 0-5, output bits 6-12 on state bits
    a..a+6 and the tile index on the bits between and above; the view
    covers 2^L amplitudes and each box lies inside it.  Reordered staging
    tiles (4-D and 5-D views) are included."""
    n = 6
    p, _ = capi.make_params(first_layer=first)
    cnt = ctypes.c_int(64)
    a = np.zeros(64, np.int32)
    st = np.zeros(64 * 13, np.uint8)
    assert svlib.sv_host_block_layout(L, ctypes.byref(p), n, ctypes.byref(cnt),
                                      a.ctypes.data_as(capi._ip), None, None, None, None,
                                      st.ctypes.data) == 0
    P = cnt.value
    bad = ctypes.c_int(0)
    assert svlib.sv_host_store_view(L, ctypes.byref(p), n, P, ctypes.byref(bad),
                                    (ctypes.c_ulonglong * 5)(), (ctypes.c_ulonglong * 4)(),
                                    (ctypes.c_uint * 5)(), (ctypes.c_int * 4)()) == capi.SV_EINVAL
    for badL, badn in ((L, 5), (12, 6)):  # not a tensor-core width / too short
        assert svlib.sv_host_store_view(badL, ctypes.byref(p), badn, 0, ctypes.byref(bad),
                                        (ctypes.c_ulonglong * 5)(), (ctypes.c_ulonglong * 4)(),
                                        (ctypes.c_uint * 5)(),
                                        (ctypes.c_int * 4)()) == capi.SV_EINVAL
    s = np.arange(1 << 13, dtype=np.int64)
    restaged = 0
    for k in range(P):
        ak = int(a[k])
        spos = [int(v) for v in st[13 * k:13 * k + 13]]
        restaged += spos != list(range(13))
        rank, dims, strides, box, coord = _store_view(svlib, L, p, k)
        assert int(np.prod(dims)) == 1 << L and int(np.prod(box)) == 1 << 13
        # output index held by staging element s, and its state bits
        y = np.zeros_like(s)
        for o in range(13):
            y |= ((s >> spos[o]) & 1) << o
        x_in = np.zeros_like(s)
        for o in range(13):
            x_in |= ((y >> o) & 1) << (o if o < n else ak + o - n)
        # box indices of s, dimension 0 fastest
        idx, rest = [], s.copy()
        for d in range(rank):
            idx.append(rest % box[d])
            rest //= box[d]
        ntlo, nthi = 1 << (ak - n), 1 << (L - ak - 7)
        for t in sorted({0, min(1, ntlo * nthi - 1), ntlo * nthi - 1, (ntlo * nthi) // 3}):
            tlo, thi = t % ntlo, t // ntlo
            c = [0] * rank
            c[coord[0]] |= tlo << coord[1]
            c[coord[2]] |= thi << coord[3]
            assert all(c[d] + box[d] <= dims[d] for d in range(rank)), (k, t)
            addr = sum((c[d] + idx[d]) * strides[d] for d in range(rank))
            want = 8 * (x_in | (tlo << n) | (thi << (ak + 7)))
            np.testing.assert_array_equal(addr, want, err_msg=f"pass {k} tile {t}")
    if (L, first) in ((16, 0), (23, 0)):
        assert restaged > 0
