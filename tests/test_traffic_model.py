"""The traffic arithmetic reproduces the numbers the paper prints (Section 7)."""
import pytest

from paper_1109_6885_gb300 import traffic


def test_eq16_worked_update_rate():
    # Eq. 16: N_D = 4M, N_C = 300, 13.5 cycles/tuple at 3.3 GHz -> "about 31,350"
    r = traffic.eq16_update_rate(4_000_000, 100_000_000, 300, 13.5, 3.3e9)
    assert r == pytest.approx(31_339, abs=1)
    assert abs(r - 31_350) / 31_350 < 0.001


def test_eq17_step1a():
    assert traffic.eq17_step1a_cpt() == pytest.approx(0.3066, abs=5e-4)   # printed 0.306


def test_step1b_six_point_six():
    # Section 7.4: Eq. 9 + 10 + 15 "around 6.6 cpt"; reproduced without Eq. 9's |U'| read
    assert traffic.step1b_model_cpt() == pytest.approx(6.68, abs=0.01)
    assert traffic.step1b_model_cpt(include_unew_read=True) == pytest.approx(7.82, abs=0.01)
    # Step 1 = 0.3 + 6.6 = 6.9 cpt, within 1% of the measured 6.97 (Table 2)
    total = traffic.eq17_step1a_cpt() + traffic.step1b_model_cpt()
    assert total == pytest.approx(6.99, abs=0.02)
    assert abs(total - 6.97) / 6.97 < 0.01


def test_step2_fourteen_point_two():
    # Section 7.4: Eq. 12 at 5 B/cycle plus Eq. 13, 14 at 7 B/cycle -> "14.2"; measured 15
    v = traffic.step2_model_cpt()
    assert v == pytest.approx(14.25, abs=0.01)
    assert abs(15.0 - v) / v < 0.055


def test_eq18_cached_step2():
    v = traffic.eq18_step2_cached_cpt()
    assert v == pytest.approx(1.733, abs=1e-3)     # printed 1.73; measured 1.85 within 7%
    assert abs(1.85 - v) / 1.85 < 0.07


def test_eq1_and_component_formulas():
    assert traffic.eq1_update_rate(1000, 0.5, 1.5) == 500
    assert traffic.eq8_step1a_bytes(8, 10, 100, L=64) == 4 * 8 * 10 + 132 * 100
    assert traffic.eq13_stream_read_bytes(20, 96, 32) == 20 * 128 / 8
    assert traffic.eq14_stream_write_bytes(21, 96, 32) == 2 * 21 * 128 / 8


def test_gpu_algorithmic_bytes():
    # 100M-row column, 20-bit codes in and out, 1M-entry main dictionary, 170k delta entries
    b2 = traffic.step2_bytes(20, 20, 100_000_000, 1_000_000, 1_000_000, 170_000)
    assert b2 == 250_000_000 + 4_000_000 + 4 * 1_170_000 + 252_500_000
    assert traffic.step1_bytes(8, 10, 5, 12) == 8 * 15 + 8 * 12 + 4 * 15
