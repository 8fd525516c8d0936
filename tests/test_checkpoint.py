"""Checkpoints of the state and the period counter (sv_save / sv_load /
sv_checkpoint_info), for resuming long evolutions (Sec. IV's 1e5-period
runs).

The CPU tests write files from the format documented in the header, with
this file's own checksum, and check that the library accepts them and
refuses damaged ones; the GPU tests resume an evolution from a checkpoint
and compare it with the uninterrupted one, bit for bit."""
import ctypes
import struct

import numpy as np
import pytest

from paper_2111_08044_gb300 import capi, inputs

FNV_BASIS = 14695981039346656037
FNV_PRIME = 1099511628211


def _fnv_words(data: bytes) -> int:
    h = FNV_BASIS
    for (w,) in struct.iter_unpack("<Q", data):
        h = ((h ^ w) * FNV_PRIME) & 0xFFFFFFFFFFFFFFFF
    return h


def _write(path, L, precision, period, payload: bytes, payload_sum=None):
    head = b"FLQSVCK1" + struct.pack("<iiqQQ", L, precision, period, len(payload),
                                     _fnv_words(payload) if payload_sum is None else payload_sum)
    head += struct.pack("<Q", _fnv_words(head))
    with open(path, "wb") as f:
        f.write(head + payload)


def _info(svlib, path):
    L, prec, per = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    rc = svlib.sv_checkpoint_info(str(path).encode(), ctypes.byref(L), ctypes.byref(prec),
                                  ctypes.byref(per))
    return rc, (L.value, prec.value, per.value)


def test_checkpoint_format_round_trip_on_host(svlib, tmp_path):
    rng = np.random.default_rng(5)
    for L, prec, dtype in ((6, capi.SV_C64, np.complex64), (5, capi.SV_C128, np.complex128),
                           (4, capi.SV_DF64, np.complex128)):
        psi = (rng.standard_normal(1 << L) + 1j * rng.standard_normal(1 << L)).astype(dtype)
        p = tmp_path / f"ok{L}.ckpt"
        _write(p, L, prec, 1234, psi.tobytes())
        assert _info(svlib, p) == (capi.SV_OK, (L, prec, 1234))


def test_checkpoint_damage_is_refused(svlib, tmp_path):
    psi = np.arange(1 << 7, dtype=np.complex64)
    good = tmp_path / "good.ckpt"
    _write(good, 7, capi.SV_C64, 3, psi.tobytes())
    raw = good.read_bytes()
    cases = {
        "payload bit": raw[:100] + bytes([raw[100] ^ 1]) + raw[101:],
        "header bit": raw[:17] + bytes([raw[17] ^ 4]) + raw[18:],
        "magic": b"X" + raw[1:],
        "truncated": raw[:-8],
        "trailing": raw + b"\0" * 8,
    }
    for name, blob in cases.items():
        p = tmp_path / f"bad_{name.replace(' ', '_')}.ckpt"
        p.write_bytes(blob)
        assert _info(svlib, p)[0] == capi.SV_EINVAL, name
    # a header whose payload size does not match L and precision
    p = tmp_path / "size.ckpt"
    _write(p, 8, capi.SV_C64, 0, psi.tobytes())
    assert _info(svlib, p)[0] == capi.SV_EINVAL
    assert _info(svlib, tmp_path / "missing.ckpt")[0] == capi.SV_EINVAL
    assert svlib.sv_save(None, b"x") == capi.SV_EINVAL
    assert svlib.sv_load(None, b"x") == capi.SV_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("precision,mode", [("c64", "block"), ("c64", "plain"), ("c128", "plain")])
def test_resume_from_checkpoint_is_bit_exact(svlib, tmp_path, precision, mode):
    from paper_2111_08044_gb300.sim import FloquetSimulator, chain_params
    cfg = inputs.ChainConfig(L=16, seed=12)
    kw = chain_params(cfg)
    if mode == "block":
        kw.update(mode=capi.SV_MODE_BLOCK, block_n=6, split=capi.SV_SPLIT_BF16X3,
                  renorm_every=3)
    path = tmp_path / "run.ckpt"
    with FloquetSimulator(cfg.L, precision=precision) as sim:
        sim.init_product_state(cfg.spinors())
        sim.build(**kw)
        sim.evolve(5)
        sim.save(path)
        e_a, n_a = sim.evolve(7)
        psi_a = sim.host_state()
    assert _info(svlib, path) == (capi.SV_OK, (cfg.L, capi.SV_C128 if precision == "c128"
                                                else capi.SV_C64, 5))
    with FloquetSimulator(cfg.L, precision=precision) as sim:
        sim.load(path)
        assert sim.period == 5
        sim.build(**kw)
        e_b, n_b = sim.evolve(7)
        psi_b = sim.host_state()
    np.testing.assert_array_equal(e_a, e_b)
    np.testing.assert_array_equal(n_a, n_b)
    np.testing.assert_array_equal(psi_a, psi_b)
    # the other precision's context refuses the file
    with FloquetSimulator(cfg.L, precision="c128" if precision == "c64" else "c64") as sim:
        with pytest.raises(capi.SvError):
            sim.load(path)
