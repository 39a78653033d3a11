"""The pins reject plausible mistakes (CPU only).

Each case copies the oracle source, plants one mistake of the kind a reader
might make when transcribing the paper (a dropped term, a wrong sign, a wrong
index or order, a transposed weight), compiles the copy, routes the oracle
wrappers through it and checks that at least one named pin now fails.
"""
import os

import pytest

import oracle
import test_oracle_basket as basket
import test_oracle_cpw as cpw
import test_oracle_lead as lead
import test_oracle_paths as paths
import test_oracle_sobol as sob

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "qmccpw_oracle.c")

MUTANTS = {
    "lookback vega divided by d": (
        "X = best;\n        D = dbest;", "X = best;\n        D = dbest / d;",
        lambda o: cpw.test_point_greeks_equal_finite_differences_of_G(o, 2, 8, 0)),
    "shifted survival term uses psi + a": (
        "const double sf_shift = norm_sf(psi - a);", "const double sf_shift = norm_sf(psi + a);",
        lambda o: cpw.test_point_value_equals_quadrature_over_first_gaussian(o, 0, 5, 0)),
    "switch point without the drift term": (
        "(log(c->K) - log(X) - omega * t1) / a", "(log(c->K) - log(X)) / a",
        lambda o: cpw.test_point_value_equals_quadrature_over_first_gaussian(o, 1, 8, 0)),
    "binary gamma sign": (
        "(psi / a - 1.0)", "(psi / a + 1.0)",
        lambda o: cpw.test_point_greeks_equal_finite_differences_of_G(o, 1, 5, 0)),
    "arithmetic vega without the strike term": (
        "out[2] = disc1 * sf_shift * D + disc * c->K * pdf * sqrt(t1);", "out[2] = disc1 * sf_shift * D;",
        lambda o: cpw.test_point_greeks_equal_finite_differences_of_G(o, 0, 8, 1)),
    "bridge weights transposed": (
        "((sr - sm) * W[l] + (sm - sl) * W[r])", "((sm - sl) * W[l] + (sr - sm) * W[r])",
        lambda o: paths.test_bridge_covariance(o, 7)),
    "bridge level filled right to left": (
        "ql[tail] = l; qr[tail] = m; ++tail;\n        ql[tail] = m; qr[tail] = r; ++tail;",
        "ql[tail] = m; qr[tail] = r; ++tail;\n        ql[tail] = l; qr[tail] = m; ++tail;",
        lambda o: paths.test_bridge_order_terminal_then_midpoints(o)),
    "pca eigenvalue index 2k+1": (
        "double s = sin((2.0 * k - 1.0) * pi / (2.0 * (2.0 * n + 1.0)));",
        "double s = sin((2.0 * k + 1.0) * pi / (2.0 * (2.0 * n + 1.0)));",
        lambda o: paths.test_pca_factor(o, 15)),
    "sobol recurrence missing the trailing m_{i-q}": (
        "        mi ^= m[i - q];\n", "",
        lambda o: sob.test_direction_integers_odd_and_bounded(o)),
    "scramble matrix upper instead of lower triangular": (
        "rows[i - 1] = (draw & above) | diag;", "rows[i - 1] = (draw & ~above & (diag - 1u)) | diag;",
        lambda o: sob.test_net_quality_first_dimensions(o, True)),
    "estimator uses natural instead of Gray index": (
        "        uint64_t index = k ^ (k >> 1);\n        for (int j = 0; j < n; ++j) {",
        "        uint64_t index = k;\n        for (int j = 0; j < n; ++j) {",
        lambda o: paths.test_estimator_points_use_the_pinned_pieces(o, 0, 16, 0)),
    "uniform without the half-ulp offset": (
        "double u = ((double)y + 0.5) * 0x1p-32;", "double u = ((double)y + 1.0) * 0x1p-32;",
        lambda o: paths.test_estimator_points_use_the_pinned_pieces(o, 2, 33, 0)),
    "standard error with R*R": (
        "se[g] = sqrt(neumaier_value(&dev) / ((double)R * (double)(R - 1)));",
        "se[g] = sqrt(neumaier_value(&dev) / ((double)R * (double)R));",
        lambda o: cpw.test_estimator_matches_geometric_asian_closed_form(o, 0, 100.0)),
    "geometric mean missing the drift": (
        "lsum += omega * s + c->sigma * W[i];", "lsum += c->sigma * W[i];",
        lambda o: cpw.test_estimator_matches_geometric_asian_closed_form(o, 1, 90.0)),
    "standard construction increments scaled by dt instead of sqrt(dt)": (
        "for (int i = 1; i <= n; ++i) W[i] = W[i - 1] + h * z[i - 1];",
        "for (int i = 1; i <= n; ++i) W[i] = W[i - 1] + dt * z[i - 1];",
        lambda o: paths.test_forward_covariance_and_structure(o, 15)),
    "standard construction driven by the dimensions in reverse": (
        "for (int i = 1; i <= n; ++i) W[i] = W[i - 1] + h * z[i - 1];",
        "for (int i = 1; i <= n; ++i) W[i] = W[i - 1] + h * z[n - i];",
        lambda o: paths.test_forward_covariance_and_structure(o, 15)),
    "leading-coordinate call vega without its density term": (
        "* phi_bar(x - b[j]) + a[j] * norm_pdf(x - b[j]));", "* phi_bar(x - b[j]));",
        lambda o: lead.test_lead_greeks_equal_finite_differences(o, 0, 5, 3)),
    "leading-coordinate binary gamma without the curvature term": (
        "(x * K - 2.0 * X1 + K * X2 / X1)", "(x * K - 2.0 * X1)",
        lambda o: lead.test_lead_greeks_equal_finite_differences(o, 1, 7, 4)),
    "leading-coordinate loading read from the second PCA column": (
        "a[j] = A[(size_t)j * (size_t)d];", "a[j] = A[(size_t)j * (size_t)d + 1];",
        lambda o: lead.test_lead_value_equals_quadrature_over_the_leading_coordinate(o, 0, 7, 4)),
    "basket loading of x_1 without the correlation": (
        "bb[i] = sig[i] * Li[0] * st1;", "bb[i] = sig[i] * st1;",
        lambda o: basket.test_basket_point_equals_quadrature_over_first_increment(o, 0, 5, 3)),
    "basket vega without the relative volatility": (
        "V += b->v[i] * exp(0.5 * bb[i] * bb[i])", "V += exp(0.5 * bb[i] * bb[i])",
        lambda o: basket.test_basket_greeks_equal_finite_differences(o, 0, 4, 3)),
    "basket binary vega without the switch-point term": (
        "(D[i] + C[i] * l1 * x)", "(D[i])",
        lambda o: basket.test_basket_greeks_equal_finite_differences(o, 1, 4, 3)),
    "basket bridge nodes read factor-major": (
        "zk[bnode] = z[bnode * m + k];", "zk[bnode] = z[k * n + bnode];",
        lambda o: basket.test_sobol_layout_of_the_basket(o)),
    "inverse normal Halley step with the wrong sign": (
        "z -= step;", "z += step;",
        lambda o: paths.test_inverse_normal_published_quantiles(o)),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_rejects_planted_mistake(tmp_path, oracle_lib, name):
    before, after, pin = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation anchor not unique: {name}"
    mutant_src = tmp_path / "mutant.c"
    mutant_src.write_text(src.replace(before, after))
    so = oracle.compile_source(str(mutant_src), str(tmp_path / "libmutant.so"))
    with oracle.using_library(so):
        with pytest.raises(AssertionError):
            pin(oracle)
    # and the unmutated oracle passes the same pin
    pin(oracle)
