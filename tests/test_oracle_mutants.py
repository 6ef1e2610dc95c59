"""Plants one plausible mistake at a time in a copy of the oracle's C source
(on the CPU) and checks that at least one pin fails on each mutant. This is
the evidence that the pins constrain every step of the oracle."""
import os

import pytest

import oracle
import oracle_pins

# (name, original text, mutated text)
MUTANTS = [
    ("ci4_nibble_order", "const unsigned nib = (idx % 2 == 0) ? (byte >> 4) : (byte & 15u);",
     "const unsigned nib = (idx % 2 == 0) ? (byte & 15u) : (byte >> 4);"),
    ("ci4_sign", "return (nib >= 8) ? (double)nib - 16.0 : (double)nib;", "return (double)nib;"),
    ("flags_ignored", "const double w = flags ? flags[(size_t)n * S + s] : 1.0;", "const double w = 1.0;"),
    ("counts_one_station", "c += (flags ? flags[(size_t)i * S + s] : 1.0) * (flags ? flags[(size_t)j * S + s] : 1.0);",
     "c += (flags ? flags[(size_t)i * S + s] : 1.0);"),
    ("dft_sign", "wim[r] = -sin(TWO_PI * r / C);", "wim[r] = sin(TWO_PI * r / C);"),
    ("fir_tap_order", "const double h = taps[(size_t)k * C + c];",
     "const double h = taps[(size_t)(T - 1 - k) * C + c];"),
    ("fir_sample_index", "const size_t t = (size_t)(s + k) * C + c;",
     "const size_t t = (size_t)(s + T - 1 - k) * C + c;"),
    ("no_channel_shift", "const int k = (m + C / 2) % C;", "const int k = m;"),
    ("delay_sign", "const double rre = b * cos(phi), rim = b * sin(phi);",
     "const double rre = b * cos(phi), rim = -b * sin(phi);"),
    ("delay_interp", "const double tau = tau_begin[n] + (tau_end[n] - tau_begin[n]) * s / S;",
     "const double tau = tau_begin[n] + (tau_end[n] - tau_begin[n]) * s / (S - 1);"),
    ("channel_freq", "return centres[sb] + (double)(k - C / 2) * fs / C;",
     "return centres[sb] + (double)k * fs / C;"),
    ("bandpass_dropped", "const double b = bandpass ? bandpass[(size_t)n * C + k] : 1.0;",
     "const double b = 1.0;"),
    ("gain_conjugated", "const double xgim = x[0] * gim + x[1] * gre;",
     "const double xgim = -x[0] * gim + x[1] * gre;"),
    ("correlate_conj", "vim += aim * bre - are * bim;", "vim += are * bim - aim * bre;"),
    ("correlate_pol_order",
     "double *v = vis + ((((size_t)sb * C + k) * B + b) * 4 + (2 * p + q)) * 2;",
     "double *v = vis + ((((size_t)sb * C + k) * B + b) * 4 + (2 * q + p)) * 2;"),
    ("baseline_index", "const size_t b = (size_t)j * (j + 1) / 2 + i;\n                    for (int p",
     "const size_t b = (size_t)j * (j + 1) / 2 + (j - i);\n                    for (int p"),
    ("vjp_drops_second_gain", "my_gg[((size_t)j * P + q) * 2] += Gre * d2re + Gim * d2im;", ""),
    ("vjp_tau_sign", "my_gt[j] -= Gre * dtre + Gim * dtim;", "my_gt[j] += Gre * dtre + Gim * dtim;"),
    ("vjp_imag_gain_sign", "my_gg[((size_t)i * P + p) * 2 + 1] += Gre * (-d1im) + Gim * d1re;",
     "my_gg[((size_t)i * P + p) * 2 + 1] += Gre * d1im + Gim * d1re;"),
    ("vjp_interp_weights_swapped", "const double fe = (double)s / (double)S, fb = 1.0 - fe;",
     "const double fb = (double)s / (double)S, fe = 1.0 - fb;"),
    ("vjp_interp_second_end_sign", "my_te[j] -= fe * t;", "my_te[j] += fe * t;"),
    ("vjp_interp_gain_conj", "const double d1r = Ur[ua] * ybr + Ui[ua] * ybi, d1i = Ui[ua] * ybr - Ur[ua] * ybi;",
     "const double d1r = Ur[ua] * ybr - Ui[ua] * ybi, d1i = Ui[ua] * ybr + Ur[ua] * ybi;"),
    ("beam_phase_sign", "const double wre = a * cos(phi), wim = a * sin(phi);",
     "const double wre = a * cos(phi), wim = -a * sin(phi);"),
    ("beam_weight_dropped", "const double a = weights ? weights[n] : 1.0;", "const double a = 1.0;"),
    ("beam_pol_swap", "const double *y = corr + (((((size_t)sb * C + k) * S + s) * N + n) * P + p) * 2;\n"
     "                                bx[p][0]",
     "const double *y = corr + (((((size_t)sb * C + k) * S + s) * N + n) * P + (1 - p)) * 2;\n"
     "                                bx[p][0]"),
    ("stokes_v_sign", "acc[3] += 2.0 * cim;", "acc[3] -= 2.0 * cim;"),
    ("stokes_u_from_imag", "acc[2] += 2.0 * cre;", "acc[2] += 2.0 * cim;"),
    ("stokes_q_sign", "acc[1] += xx - yy;", "acc[1] += yy - xx;"),
    ("stokes_tint_index", "const int s = so * tint + t;", "const int s = so + t * SO;"),
    ("incoherent_weight_squared", "acc[0] += wn * (xx + yy);", "acc[0] += wn * wn * (xx + yy);"),
    ("incoherent_u_sign", "acc[2] += wn * 2.0 * (xre * yre + xim * yim);    /* 2 Re(X conj Y) */",
     "acc[2] += wn * 2.0 * (xre * yre - xim * yim);    /* 2 Re(X conj Y) */"),
    ("incoherent_one_station", "const double *y = corr + ((((size_t)sb * C + k) * S + s) * N + n) * P * 2;",
     "const double *y = corr + ((((size_t)sb * C + k) * S + s) * N + 0) * P * 2;"),
]


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, orig, mut):
    src = open(oracle.SOURCE).read()
    assert src.count(orig) == 1, f"mutation site for {name} not unique"
    path = os.path.join(tmp_path, "fx_oracle_mut.c")
    with open(path, "w") as f:
        f.write(src.replace(orig, mut))
    lib = oracle.compile_oracle(path, os.path.join(tmp_path, "libmut.so"))
    o = oracle.Oracle(lib)
    failed = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(o)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught mutant {name}"
