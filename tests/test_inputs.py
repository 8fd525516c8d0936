"""Seeded input generator: SplitMix64 against its published outputs."""
import numpy as np

from paper_2111_08044_gb300 import inputs


def test_splitmix64_reference_outputs():
    r = inputs.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4
    r = inputs.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_spinors_normalised_and_angles_in_range():
    ang = inputs.bloch_angles(inputs.SplitMix64(5), 30)
    assert np.all((ang[:, 0] >= 0) & (ang[:, 0] <= np.pi))
    assert np.all((ang[:, 1] >= 0) & (ang[:, 1] < 2 * np.pi))
    sp = inputs.spinors_from_angles(ang)
    np.testing.assert_allclose((sp ** 2).sum(axis=1), 1.0, atol=1e-15)


def test_batch_preset_ranges():
    chains = inputs.batch_preset(64)
    Ls = [c.L for c in chains]
    assert min(Ls) >= 14 and max(Ls) <= 22
    for c in chains:
        assert 0.8 <= c.J <= 1.2 and 0.6 <= c.hx <= 1.0
        assert 0.2 <= c.hz <= 0.6 and 0.1 <= c.theta <= 0.5
    assert inputs.batch_preset(64)[7].seed == chains[7].seed
