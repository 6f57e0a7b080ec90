"""The pins discriminate: plausible mistakes planted in a copy of the oracle
source (on the CPU, in a temporary directory) each fail at least one pin.

The committed oracle is never modified; every mutant is a text substitution
on a temporary copy, compiled and loaded in place of the real build for the
duration of one check.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_cells as cpins
import test_oracle_edge as epins
import test_oracle_variants as vpins

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
    ("divergent-flow term takes 1/2 instead of 1/4",
     "return -quarter * C * (D(L) + D(R)) / (half * (G[L] + G[R]));",
     "return -half * C * (D(L) + D(R)) / (half * (G[L] + G[R]));"),
    ("divergent-flow term not divided by the face G",
     "return -quarter * C * (D(L) + D(R)) / (half * (G[L] + G[R]));",
     "return -quarter * C * (D(L) + D(R));"),
    ("divergent-flow divergence drops the V difference",
     "return (u[c] - u[c - X]) + (v[c] - v[c - Y]) + (w[c] - w[c - Z]);",
     "return (u[c] - u[c - X]) + (w[c] - w[c - Z]);"),
    ("divergent-flow divergence drops the W difference",
     "return (u[c] - u[c - X]) + (v[c] - v[c - Y]) + (w[c] - w[c - Z]);",
     "return (u[c] - u[c - X]) + (v[c] - v[c - Y]);"),
    ("infinite gauge cross numerator takes 1/4",
     "const T n1 = eighth * (P[R + e1]",
     "const T n1 = quarter * (P[R + e1]"),
    ("infinite gauge A loses its 1/2",
     "const T dA = half * (P[R] - P[L]);",
     "const T dA = (P[R] - P[L]);"),
    ("infinite gauge limiter takes donor fluxes",
     "auto fl = [&](T L, T R, T C) { return unit ? C : donor(L, R, C); };",
     "auto fl = [&](T L, T R, T C) { return donor(L, R, C); };"),
    ("signed limiter keeps the velocity's direction",
     "const bool flip = sgn && val(val(Ut) >= 0.0 ? P[L] : P[R]) < 0.0;",
     "const bool flip = false && sgn;"),
    ("signed variant forms A and B from psi",
     "for (long q = 0; q < n; ++q) Pa[q] = oabs(P[q]);",
     "for (long q = 0; q < n; ++q) Pa[q] = P[q];"),
    ("edge flux takes the downwind node",
     "flux[k * m.E + e] = pD[k * m.N + ip1] * zpos + pD[k * m.N + ip2] * zneg;",
     "flux[k * m.E + e] = pD[k * m.N + ip2] * zpos + pD[k * m.N + ip1] * zneg;"),
    ("vertical edge-stage flux takes the downwind level",
     "fluz[k * m.N + n] = std::max(0.0, w) * pD[(k - 1) * m.N + n] +\n"
     "                          std::min(0.0, w) * pD[k * m.N + n];",
     "fluz[k * m.N + n] = std::max(0.0, w) * pD[k * m.N + n] +\n"
     "                          std::min(0.0, w) * pD[(k - 1) * m.N + n];"),
    ("edge divergence ignores the edge signs",
     "for (int j = 0; j < 6; ++j) s += m.sgn[6 * n + j] * flux[k * m.E + m.n2e[6 * n + j]];",
     "for (int j = 0; j < 6; ++j) s += flux[k * m.E + m.n2e[6 * n + j]];"),
    ("top boundary flux copies the bottom face",
     "fluz[m.nz * m.N + n] = pivbz * fluz[(m.nz - 1) * m.N + n];",
     "fluz[m.nz * m.N + n] = pivbz * fluz[m.N + n];"),
    ("edge advance forgets rho",
     "for (long q = 0; q < m.N * m.nz; ++q) pD[q] = pD[q] - div[q] / rho[q];",
     "for (long q = 0; q < m.N * m.nz; ++q) pD[q] = pD[q] - div[q];"),
    ("edge divergence forgets the dual volume",
     "div[k * m.N + n] = s / vol[n];",
     "div[k * m.N + n] = s;"),
    ("cell sum reads the first neighbour twice",
     "B[k * ncells + s] = (a[t[s]] + a[t[ncells + s]] + a[t[2 * ncells + s]]) * fac;",
     "B[k * ncells + s] = (a[t[s]] + a[t[ncells + s]] + a[t[s]]) * fac;"),
    ("cell sum ignores its factor",
     "B[k * ncells + s] = (a[t[s]] + a[t[ncells + s]] + a[t[2 * ncells + s]]) * fac;",
     "B[k * ncells + s] = (a[t[s]] + a[t[ncells + s]] + a[t[2 * ncells + s]]);"),
    ("y halo not wrapped",
     "for (int i = -g.h; i < g.nx + g.h; ++i) f[g.at(i, j, k)] = f[g.at(i, wrap(j, g.ny), k)];",
     "for (int i = -g.h; i < g.nx + g.h; ++i) f[g.at(i, j, k)] = f[g.at(i, j < 0 ? 0 : g.ny - 1, k)];"),
]


def _pin_battery(stop_at_first: bool = False):
    """Fast pin checks, the cheapest first; each returns normally or raises.
    Returns how many failed (with stop_at_first: 0 or 1)."""
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
        lambda: pins.test_limiter_inactive_on_smooth_monotone_data("x", -0.4),
        lambda: pins.test_limiter_inactive_on_smooth_monotone_data("y", 0.4),
        lambda: pins.test_limiter_inactive_on_smooth_monotone_data("z", -0.4),
        lambda: pins.test_adjoint_dot_product_against_tlm(2, 1, 1, 0),
        lambda: pins.test_adjoint_dot_product_against_tlm(2, 0, 1, 0),
        pins.test_halo_fill_periodic_k_matches_numpy_pad,
        lambda: pins.test_courant_one_shift_vertical_periodic(2, 1, 1),
        pins.test_adjoint_dot_product_on_rotating_cone,
        lambda: epins.test_mass_conservation_closed(True),
        lambda: epins.test_courant_one_shift_along_each_colour(2, 1),
        lambda: epins.test_vertical_courant_one_shift_with_closed_ends(1),
        epins.test_open_boundaries_copy_the_adjacent_face,
        lambda: cpins.test_constant_and_total("SN"),
        lambda: cpins.test_delta_response_is_the_edge_neighbours("UN"),
        lambda: pins.test_convergence_order(2, 0, 1.9, 2.3),
        lambda: vpins.test_dfl_restores_second_order_in_divergent_flow("x", True),
        lambda: vpins.check_dfl_2d("xy", (24, 48, 96)),
        lambda: vpins.check_dfl_2d("xz", (24, 48, 96)),
        lambda: vpins.test_iga_is_the_limit_of_a_growing_gauge(1),
        lambda: vpins.test_abs_is_odd_in_psi(2, 1, 0),
        lambda: vpins.test_limited_signed_step_makes_no_new_extrema(vpins.ABS),
    ]
    failed = 0
    for chk in checks:
        try:
            chk()
        except Exception:      # an assertion, or NaN/shape trouble the mistake caused
            failed += 1
            if stop_at_first:
                break
    return failed


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    """Every mutant compiled up front, several g++ processes at a time;
    a mutant whose anchor is not found exactly once maps to None."""
    d = tmp_path_factory.mktemp("mutants")
    src = open(SRC).read()

    def build_one(idx, orig, mut):
        if src.count(orig) != 1:
            return None
        p = d / f"mutant{idx}.cpp"
        p.write_text(src.replace(orig, mut))
        return oracle.build(force=True, src=str(p), out=str(d / f"libmutant{idx}.so"))

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {name: ex.submit(build_one, i, orig, mut)
                for i, (name, orig, mut) in enumerate(MUTANTS)}
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.slow
@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, orig, mut, mutant_libs):
    assert open(SRC).read().count(orig) == 1, f"mutation anchor not unique/found: {name}"
    prev = oracle.use_library(mutant_libs[name])
    try:
        failed = _pin_battery(stop_at_first=True)
    finally:
        oracle.restore_library(prev)
    assert failed >= 1, f"no pin caught the planted mistake: {name}"


def test_unmutated_oracle_passes_battery():
    assert _pin_battery() == 0
