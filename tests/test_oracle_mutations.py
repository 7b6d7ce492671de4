"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (on the CPU, in a
temporary directory), builds it, and checks that at least one of the pins in
test_oracle_pins.py fails against the mutant. The oracle under tests/ and
oracle/ is never modified.
"""
import importlib.util
import math
import os
import shutil

import pytest

import tests.test_oracle_pins as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, mutated text): each a mistake a careful implementer
# could make reading the paper.
MUTATIONS = [
    ("reaction sign", "return val - q.r * u;", "return val + q.r * u;"),
    ("drop y in mu_r", "+ y;\n    q.muv", ";\n    q.muv"),
    ("sign of 2 kappa y in mu_y", "r2g * v - 2.0 * m->kappa * y;", "r2g * v + 2.0 * m->kappa * y;"),
    ("half of zeta_rr dropped", "q.zrr = 0.5 * m->lambda", "q.zrr = 1.0 * m->lambda"),
    ("mixed stencil divided by 2 h h", "return g3 * s / (4.0 * x->h[0] * x->h[1]);",
     "return g3 * s / (2.0 * x->h[0] * x->h[1]);"),
    ("mixed corner sign", "- U[at(x, i - 1, k + 1, j)] + U[at(x, i - 1, k - 1, j)];",
     "+ U[at(x, i - 1, k + 1, j)] - U[at(x, i - 1, k - 1, j)];"),
    ("Jacobian with sinh (the printed typo)", "*J = alpha * (c2 - c1) * cosh(a);",
     "*J = alpha * (c2 - c1) * sinh(a);"),
    ("J2 term sign in g4", "double g4 = q.mur / J - q.zrr * J2 / (J * J * J);\n            val",
     "double g4 = q.mur / J + q.zrr * J2 / (J * J * J);\n            val"),
    ("g5 divided by J^2", "double g5 = q.muv / J - q.zvv * J2 / (J * J * J);\n            return",
     "double g5 = q.muv / (J * J) - q.zvv * J2 / (J * J * J);\n            return"),
    ("theta dropped in Douglas stages", "double w = x->g.theta_adi * x->dt;", "double w = x->dt;"),
    ("Thomas uses the wrong sub-diagonal", "dp[i] = (d[i] - a[i] * dp[i - 1]) / m;",
     "dp[i] = (d[i] - a[i - 1] * dp[i - 1]) / m;"),
    ("v and y solves swapped", "orc_solve_dir(x, 1, th, a, b);\n    orc_solve_dir(x, 2, th, b, a);",
     "orc_solve_dir(x, 2, th, a, b);\n    orc_solve_dir(x, 1, th, b, a);"),
    ("Dirichlet data at t^n", "dU0[p] = orc_dirichlet(x, t1,", "dU0[p] = orc_dirichlet(x, t,"),
    ("payoff kink sign", "double rstar = log(DA) / G;\n    double mlo",
     "double rstar = -log(DA) / G;\n    double mlo"),
    ("Delta_M without the strike", "x->DM = 1.0 + (in->TM - in->T) * x->K;", "x->DM = 1.0 + (in->TM - in->T);"),
    ("readout at the wrong v", "double xv = metric_xi(x, 1, x->m.v0) / x->h[1];",
     "double xv = metric_xi(x, 1, 0.5 * x->m.v0) / x->h[1];"),
    ("forward derivative sign", "return -c->beta1 / c->tau * e + c->beta2",
     "return c->beta1 / c->tau * e + c->beta2"),
    ("one-sided face difference wrong", "(-3.0 * u0 + 4.0 * u1 - u2) / (2.0 * h)",
     "(-3.0 * u0 + 4.0 * u1 - u2) / h"),
    ("v lines read with r stride", "else if (d == 1) { *i = (int)(line % x->n[0]); *k = p;",
     "else if (d == 1) { *i = (int)(line % x->n[1]); *k = p;"),
    ("Greek without the metric Jacobian", "*d_dr = sr / (x->h[0] * Jr);", "*d_dr = sr / x->h[0];"),
    ("derivative weight sign", "double p = 1.0 / (double)(m - l);", "double p = 1.0 / (double)(l - m);"),
    ("vega from the r weights", "sv += wr[a] * dwv[b] * U[at(x, ir + a, iv + b, 0)];",
     "sv += dwr[a] * wv[b] * U[at(x, ir + a, iv + b, 0)];"),
    ("CS mixed correction with weight 1", "double c = sch == 1 ? 0.5 : theta;",
     "double c = sch == 1 ? 1.0 : theta;"),
    ("MCS mixed correction with weight 1/2", "double c = sch == 1 ? 0.5 : theta;", "double c = 0.5;"),
    ("HV correction with weight theta", "double c = sch == 2 ? 0.5 - theta : 0.5;",
     "double c = sch == 2 ? 0.5 - theta : theta;"),
    ("MCS second sweep about Y3", "(sch == 3 ? y3[p] : U[p])", "(sch >= 2 ? y3[p] : U[p])"),
    ("HV second sweep about U^n",
     "if (sch == 3)\n        for (long p = 0; p < N; ++p) z[p] -= a[p];",
     "if (sch == 4)\n        for (long p = 0; p < N; ++p) z[p] -= a[p];"),
    ("CS family explicit operators at t^n", "int mid = x->g.explicit_midpoint || x->g.scheme != 0;",
     "int mid = x->g.explicit_midpoint;"),
    ("spline right-hand side halved", "double d = 6.0 * ((sp->y[i + 1] - sp->y[i]) / hr",
     "double d = 3.0 * ((sp->y[i + 1] - sp->y[i]) / hr"),
    ("spline end slope sign", "+ h / 6.0 * (sp->M[m - 2] + 2.0 * sp->M[m - 1]);",
     "- h / 6.0 * (sp->M[m - 2] + 2.0 * sp->M[m - 1]);"),
    ("spline last interval never used", "while (i < m - 2 && t >= sp->tau[i + 1]) ++i;",
     "while (i < m - 3 && t >= sp->tau[i + 1]) ++i;"),
    ("knot forward sign", "        knot_curve_at(c, t, &s, &ds, &d2s);\n        return -ds;",
     "        knot_curve_at(c, t, &s, &ds, &d2s);\n        return ds;"),
    ("knot drift curvature sign in the PDE", "        df0 = -d2s;", "        df0 = d2s;"),
    ("floorlet integral over the whole cell",
     "double integral = DA * exp(-G * ra) * (-expm1(-G * (mhi - ra))) / G - (mhi - ra);",
     "double integral = DA * exp(-G * ra) * (-expm1(-G * (mhi - ra))) / G - (rb - ra);"),
    ("floorlet paid on the caplet side", "double mhi = rb < rstar ? rb : rstar;", "double mhi = rb;"),
]


def _load_mutant(tmp_path, name, old, new):
    src = open(os.path.join(ROOT, "oracle", "hjm_oracle.c")).read()
    assert src.count(old) == 1, "mutation anchor not unique: %s" % name
    d = tmp_path / "oracle_mut"
    d.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), d / "__init__.py")
    shutil.copy(os.path.join(ROOT, "oracle", "hjm_oracle.h"), d / "hjm_oracle.h")
    (d / "hjm_oracle.c").write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle_mut_%d" % abs(hash(name)), d / "__init__.py",
                                                  submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


def _pins(orc):
    """A fast subset of the pins, as callables on an oracle module."""
    yield lambda: P.test_discount_is_exp_minus_integral_of_forward(orc, P.W.ns_curve(0.03, -0.01, 0.015, 2.0))
    for g in (0.0, 0.9):
        for name in ("r2", "v2", "y", "rv", "mix"):
            yield lambda g=g, name=name: P.test_operator_exact_on_quadratics(orc, g, name)
    yield lambda: P.test_operator_second_order_on_sinh_grid(orc)
    yield lambda: P.test_metric_jacobians_are_derivatives_of_the_map(orc)
    yield lambda: P.test_implicit_rows_reproduce_operator(orc, 0.0)
    for d in range(3):
        yield lambda d=d: P.test_line_solves_equal_dense_lu(orc, d)
    yield lambda: P.test_douglas_step_equals_dense_product(orc, 1)
    yield lambda: P.test_dirichlet_data(orc)
    yield lambda: P.test_payoff_average_exact_in_r(orc)
    yield lambda: P.test_floorlet_payoff_average_exact_in_r(orc)
    yield lambda: P.test_readout_exact_on_bicubics(orc)
    yield lambda: P.test_greeks_exact_on_bicubics(orc)
    yield lambda: P.test_config1_bond_price(orc)
    yield lambda: P.test_bond_ns_curve_converges(orc)
    yield lambda: P.test_gaussian_limit_converges_to_closed_form(orc, P.W.flat_curve(0.03))
    yield lambda: P.test_knot_curve_interpolates_the_knots(orc)
    yield lambda: P.test_knot_curve_of_a_flat_curve_is_flat(orc)
    yield lambda: P.test_knot_curve_is_the_natural_cubic_spline_of_ln_p(orc)
    yield lambda: P.test_knot_curve_continues_flat_past_the_last_knot(orc)
    yield lambda: P.test_knot_curve_bond_reprices_the_curve(orc)
    yield lambda: P.test_craig_sneyd_reductions(orc)
    for sch in range(4):
        yield lambda sch=sch: P.test_craig_sneyd_family_time_order(orc, sch)
    yield lambda: P.test_craig_sneyd_family_second_order_with_time_dependent_drift(orc, 1)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(tmp_path, name, old, new):
    mut = _load_mutant(tmp_path, name, old, new)
    for pin in _pins(mut):
        try:
            pin()
        except Exception:  # an assertion, a rejected input or a numerical failure
            return
    pytest.fail("no pin caught the planted mistake: %s" % name)


def test_unmutated_copy_passes_the_same_pins(tmp_path):
    mut = _load_mutant(tmp_path, "identity", "static const double ORC_PI", "static const double ORC_PI")
    for pin in _pins(mut):
        pin()
    assert math.isfinite(mut.price(P.W.config1()))
