"""The pins discriminate: plausible mistakes planted in a copy of the oracle
source (on the CPU, in a temporary directory) each fail at least one pin.

The committed oracle is never modified; every mutant is a text substitution
on a temporary copy, compiled and loaded in place of the real build for the
duration of one check.
"""
import os
import tempfile

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "mpdata_oracle.cpp")

# (name, original text, planted mistake)
MUTANTS = [
    ("cross term loses its 1/2",
     "T By = half * (P[R + Y] + P[L + Y] - P[R - Y] - P[L - Y]) /\n"
     "                 (P[R + Y] + P[L + Y] + P[R - Y] + P[L - Y] + eps);\n          T Bz",
     "T By = (P[R + Y] + P[L + Y] - P[R - Y] - P[L - Y]) /\n"
     "                 (P[R + Y] + P[L + Y] + P[R - Y] + P[L - Y] + eps);\n          T Bz"),
    ("cross term sign flipped",
     "ut[c] = (oabs(U) - U * U / Gf) * A - U * (Vb * By + Wb * Bz) / Gf;",
     "ut[c] = (oabs(U) - U * U / Gf) * A + U * (Vb * By + Wb * Bz) / Gf;"),
    ("G dropped from |U| - U^2/G",
     "ut[c] = (oabs(U) - U * U / Gf) * A",
     "ut[c] = (oabs(U) - U * U) * A"),
    ("A ratio reversed",
     "vt[c] = (oabs(V) - V * V / Gf) * A",
     "vt[c] = (oabs(V) - V * V / Gf) * (-A)"),
    ("cross average takes the wrong row",
     "T Vb = quarter * (v[L] + v[R] + v[L - Y] + v[R - Y]);\n          T Wb",
     "T Vb = quarter * (v[L] + v[R] + v[L + Y] + v[R + Y]);\n          T Wb"),
    ("vertical cross term uses U for V",
     "T Vb = quarter * (v[L] + v[R] + v[L - Y] + v[R - Y]);\n          wt[c]",
     "T Vb = quarter * (u[L] + u[R] + u[L - Y] + u[R - Y]);\n          wt[c]"),
    ("upwind operands transposed",
     "return omax(C, T(0.0)) * L + omin(C, T(0.0)) * R;",
     "return omax(C, T(0.0)) * R + omin(C, T(0.0)) * L;"),
    ("beta-up uses the outgoing sum",
     "bu[c] = (hi - P[c]) * G[c] / (in + eps);",
     "bu[c] = (hi - P[c]) * G[c] / (out + eps);"),
    ("limited face swaps donor and receiver",
     "T cpos = omin(omin(one, bdL), buR);",
     "T cpos = omin(omin(one, buL), bdR);"),
    ("limiter bounds miss the upward neighbour",
     "const long nb[6] = {-X, X, -Y, Y, -Z, Z};\n#pragma omp parallel for",
     "const long nb[6] = {-X, -X, -Y, Y, -Z, Z};\n#pragma omp parallel for"),
    ("top face left open",
     "  if (g.kper) return;  // periodic k: every face is open, the halo wraps\n  for (int k = -g.h; k < g.nz + g.h; ++k) {\n    if (k >= 0 && k < g.nz - 1) continue;",
     "  if (g.kper) return;  // periodic k: every face is open, the halo wraps\n  for (int k = -g.h; k < g.nz + g.h; ++k) {\n    if (k >= 0 && k < g.nz) continue;"),
    ("advance forgets 1/G",
     "out[c] = P[c] - ((fxp - fxm) + (fyp - fym) + (fzp - fzm)) / G[c];",
     "out[c] = P[c] - ((fxp - fxm) + (fyp - fym) + (fzp - fzm));"),
    ("epsilon dropped",
     "const double EPS = 1e-15;",
     "const double EPS = 0.0;"),
    ("adjoint drops the 1/4 of the cross average",
     "c1b[L] += 0.25 * C1b; c1b[R] += 0.25 * C1b;",
     "c1b[L] += C1b; c1b[R] += 0.25 * C1b;"),
    ("adjoint routes the limiter factor to the wrong beta",
     "if (p_first) { if (p_is_bdL) *bdLb += cpb; } else { *buRb += cpb; }",
     "if (p_first) { if (p_is_bdL) *buRb += cpb; } else { *bdLb += cpb; }"),
    ("adjoint skips folding the psi1 halo",
     "    rev_halo_periodic(Pb.data(), g);  // the pass's input state had its halo filled\n",
     "\n"),
    ("adjoint breaks bound ties the other way",
     "if (!(hi >= P[c])) { hi = P[c]; hip = &Pb[c]; }",
     "if (!(hi > P[c])) { hi = P[c]; hip = &Pb[c]; }"),
    ("adjoint forgets d|U|/dU",
     "*Ub += ub * (sg * A - 2.0 * U / Gf * A - X / Gf);",
     "*Ub += ub * (-2.0 * U / Gf * A - X / Gf);"),
    ("periodic k halo copies the edge level",
     "int ks = g.kper ? wrap(k, g.nz) : (k < 0 ? 0 : g.nz - 1);\n    for (int j = -g.h; j < g.ny + g.h; ++j)\n      for (int i = -g.h; i < g.nx + g.h; ++i) f[",
     "int ks = (k < 0 ? 0 : g.nz - 1);\n    for (int j = -g.h; j < g.ny + g.h; ++j)\n      for (int i = -g.h; i < g.nx + g.h; ++i) f["),
    ("y halo not wrapped",
     "for (int i = -g.h; i < g.nx + g.h; ++i) f[g.at(i, j, k)] = f[g.at(i, wrap(j, g.ny), k)];",
     "for (int i = -g.h; i < g.nx + g.h; ++i) f[g.at(i, j, k)] = f[g.at(i, j < 0 ? 0 : g.ny - 1, k)];"),
]


def _pin_battery():
    """Fast pin checks; each returns normally or raises."""
    checks = [
        pins.test_halo_fill_matches_numpy_pad,
        lambda: pins.test_donor_cell_fourier_1d(0.3, 1.0, "x"),
        lambda: pins.test_donor_cell_fourier_1d(-0.45, 1.0, "y"),
        lambda: pins.test_donor_cell_fourier_1d(0.7, 2.0, "x"),
        pins.test_donor_cell_fourier_2d,
        pins.test_mpdata_linearised_symbol_1d,
        lambda: pins.test_mass_conservation(2, 1),
        lambda: pins.test_constant_preservation(5),
        lambda: pins.test_courant_one_shift_horizontal(2, 1, "x", 1),
        lambda: pins.test_courant_one_shift_horizontal(2, 1, "y", -1),
        lambda: pins.test_courant_one_shift_vertical_zero_flux(2, 1),
        lambda: pins.test_pseudo_velocity_taylor_limit(False),
        lambda: pins.test_pseudo_velocity_taylor_limit(True),
        pins.test_limiter_monotone_rotating_cone,
        pins.test_limiter_monotone_step_3d,
        lambda: pins.test_positivity(0),
        lambda: pins.test_positivity(1),
        lambda: pins.test_convergence_order(2, 0, 1.9, 2.3),
        lambda: pins.test_limiter_inactive_on_smooth_monotone_data("x", -0.4),
        lambda: pins.test_limiter_inactive_on_smooth_monotone_data("y", 0.4),
        lambda: pins.test_limiter_inactive_on_smooth_monotone_data("z", -0.4),
        lambda: pins.test_adjoint_dot_product_against_tlm(2, 1, 1, 0),
        lambda: pins.test_adjoint_dot_product_against_tlm(2, 0, 1, 0),
        pins.test_halo_fill_periodic_k_matches_numpy_pad,
        lambda: pins.test_courant_one_shift_vertical_periodic(2, 1, 1),
        pins.test_adjoint_dot_product_on_rotating_cone,
    ]
    failed = 0
    for chk in checks:
        try:
            chk()
        except Exception:      # an assertion, or NaN/shape trouble the mistake caused
            failed += 1
    return failed


@pytest.mark.slow
@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, orig, mut):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation anchor not unique/found: {name}"
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "mutant.cpp")
        with open(p, "w") as f:
            f.write(src.replace(orig, mut))
        lib = oracle.build(force=True, src=p, out=os.path.join(d, "libmutant.so"))
        prev = oracle.use_library(lib)
        try:
            failed = _pin_battery()
        finally:
            oracle.restore_library(prev)
    assert failed >= 1, f"no pin caught the planted mistake: {name}"


def test_unmutated_oracle_passes_battery():
    assert _pin_battery() == 0
