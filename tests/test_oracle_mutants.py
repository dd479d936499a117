"""Planted mistakes in the oracle must be caught by its pins.

Each case copies lv_oracle.c, plants one plausible mistake (a dropped term,
a wrong sign, a wrong index, a swapped operand), compiles the copy on the
CPU and runs the pin battery against it: at least one pin has to fail.
This checks that the pins are strong enough to vouch for the oracle.
"""
import os

import pytest

import oracle

from . import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "lv_oracle.c")

MUTANTS = {
    "drift sign": ("            x[n + 1] = x[n] + (op->r - 0.5 * pt.sigma * pt.sigma) * dt",
                   "            x[n + 1] = x[n] + (op->r + 0.5 * pt.sigma * pt.sigma) * dt"),
    "dx/dsigma sign": ("double h = on_x ? x[n] * sqdt * z[n] : sqdt * z[n] - pt.sigma * dt;",
                       "double h = on_x ? x[n] * sqdt * z[n] : sqdt * z[n] + pt.sigma * dt;"),
    "dsigma/dx drops S": ("factor = 1.0 + h * S * pt.dsigma_dS;",
                          "factor = 1.0 + h * pt.dsigma_dS;"),
    "node weights transposed": ("p->w[1] = u * (1.0 - v);", "p->w[1] = (1.0 - u) * v;"),
    "philox wrong product": ("uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi0 ^ c1 ^ k0;"),
    "philox key schedule": ("k1 += ORC_PHILOX_W1;", "k1 += ORC_PHILOX_W0;"),
    "box-muller cos/sin swapped": ("z[2 * pair] = radius * cos(angle);",
                                   "z[2 * pair] = radius * sin(angle);"),
    "uniform offset dropped": ("((double)(w >> 9) + 0.5)", "((double)(w >> 9) + 0.0)"),
    "discount missing in adjoint": ("disc * (double)op->phi * (on_x ? 1.0 : SN) : 0.0",
                                    "(double)op->phi * (on_x ? 1.0 : SN) : 0.0"),
    "time-neighbour index": ("double s01 = (J > 1) ? sf->sigma[i * J + j + 1] : 0.0;",
                             "double s01 = (J > 1) ? sf->sigma[i * J + j] : 0.0;"),
    "cell rule strict": ("if (nodes[mid] <= x) lo = mid;", "if (nodes[mid] < x) lo = mid;"),
    "slope kept outside grid": ("if (inside)\n", "if (1)\n"),
    "sigma at right point": ("double t = (double)n * dt;\n        double S = on_x ? x[n] : exp(x[n]);\n"
                             "        st = orc_sigma_decided(sf, S, t, orc_forced_cell(dec, c_first, c_last, n), band, &pt, "
                             "&overridden);\n        if (st != ORC_OK) return st;\n        ov[0] += overridden;",
                             "double t = (double)(n + 1) * dt;\n        double S = on_x ? x[n] : exp(x[n]);\n"
                             "        st = orc_sigma_decided(sf, S, t, orc_forced_cell(dec, c_first, c_last, n), band, &pt, "
                             "&overridden);\n        if (st != ORC_OK) return st;\n        ov[0] += overridden;"),
    "inside test drops the upper edge": ("int inside = (S >= sf->spot[0] && S <= sf->spot[I - 1]);",
                                         "int inside = (S >= sf->spot[0]);"),
    "payoff sign": ("const double itm = (double)op->phi * (SN - op->K);\n    res->V",
                    "const double itm = (SN - op->K);\n    res->V"),
    "log-weight slope drops 1/S": ("double du_dS = logs ? 1.0 / (S * (log(hi_s) - log(lo_s)))",
                                   "double du_dS = logs ? 1.0 / (log(hi_s) - log(lo_s))"),
    "log weight taken in S": ("u = logs ? (log(S) - log(lo_s)) / (log(hi_s) - log(lo_s))",
                              "u = logs ? (S - lo_s) / (log(hi_s) - log(lo_s))"),
    "Euler on X: adjoint drops r dt": ("factor = 1.0 + op->r * dt + pt.sigma * sqdt * z[n] + h * pt.dsigma_dS;",
                                       "factor = 1.0 + pt.sigma * sqdt * z[n] + h * pt.dsigma_dS;"),
    "Euler on X: dx/dsigma drops the spot": ("double h = on_x ? x[n] * sqdt * z[n]", "double h = on_x ? sqdt * z[n]"),
    "rho drops the discount's share": ("double rho = -op->T * res->V;", "double rho = 0.0;"),
    "d V / d T: step time factor off by one": ("h * pt.dsigma_dt * (double)n / (double)N",
                                               "h * pt.dsigma_dt * (double)(n + 1) / (double)N"),
    "vanna: drops the slope term of d h / d sigma": ("sqdt * z[n] * (1.0 + kappa / (pt.sigma * f))",
                                                     "sqdt * z[n] * (1.0)"),
    "vanna: score sign": ("(z[n] * z[n] - 1.0) / pt.sigma - sqdt", "(1.0 - z[n] * z[n]) / pt.sigma - sqdt"),
    "vanna: slope term without 1 / (1 + g)": ("const double b = h / f;", "const double b = h;"),
    "vanna: weight slope sign": ("const double dw[4] = { -(1.0 - v) * pt.du_dS, (1.0 - v) * pt.du_dS,",
                                 "const double dw[4] = { (1.0 - v) * pt.du_dS, -(1.0 - v) * pt.du_dS,"),
    "vanna: delta without D_N": ("phi * SN * D / op->S0 : 0.0;", "phi * SN / op->S0 : 0.0;"),
    "d V / d T: drift term sign": ("dx_ddt = (op->r - 0.5 * pt.sigma * pt.sigma)", "dx_ddt = (op->r + 0.5 * pt.sigma * pt.sigma)"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name!r} not unique"
    src = tmp_path / "lv_oracle_mutant.c"
    src.write_text(text.replace(old, new))
    so = str(tmp_path / "liblv_oracle_mutant.so")
    oracle.build(src=str(src), out=so)
    lib = oracle.load_library(so)
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
            break
    assert caught, f"no pin caught the planted mistake {name!r}"
