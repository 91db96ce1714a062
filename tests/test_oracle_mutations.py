"""The oracle's pins are sensitive: plant a plausible mistake in one oracle
function, on the CPU, and at least one pin of tests/test_oracle_pins.py must
fail on it.

Each case wraps the real oracle in a proxy whose named function carries the
mistake: a sign, an index shifted by one, a dropped term, a wrong scale, a
transposed operand.  The pins are then run against the proxy exactly as they
run against the oracle.  A pin that calls a function through another oracle
function does not see the mistake, so every case lists the pins that call the
mutated function directly.
"""
import numpy as np
import pytest

import test_oracle_pins as pins


class Mutant:
    """The oracle with some functions replaced."""

    def __init__(self, base, **repl):
        self._base = base
        self._repl = repl

    def __getattr__(self, name):
        return self._repl[name] if name in self._repl else getattr(self._base, name)


def _wrong_phi3(r):
    # inner branch with 2 r^2 for 3 r^2
    a = abs(r)
    if a <= 0.5:
        return (1.0 + np.sqrt(1.0 - 2.0 * a * a)) / 3.0
    if a <= 1.5:
        d = 1.0 - a
        return (5.0 - 3.0 * a - np.sqrt(max(0.0, 1.0 - 3.0 * d * d))) / 6.0
    return 0.0


def _curl_with_flipped_term(o):
    def curl(u, dx=1.0):
        w = o.curl_box(u, dx).copy()
        w[0] = -w[0]
        return w
    return curl


def _transposed_source(o):
    def pd(b, src, f, tgt, **kw):
        n = np.asarray(f).shape[0]
        ft = np.asarray(f).reshape(n, b, b, b).transpose(0, 3, 2, 1).reshape(n, -1)
        return o.poisson_direct(b, src, ft, tgt, **kw)
    return pd


# (name, replacements built from the oracle, pins to run: (function, extra args))
CASES = [
    ("G_L sign", lambda o: dict(lgf_quad=lambda *n: -o.lgf_quad(*n)),
     [(pins.test_lgf_origin_watson, ()), (pins.test_far_field_leading_term, ())]),
    ("G_L Bessel order shifted by one", lambda o: dict(lgf_quad=lambda a, b, c: o.lgf_quad(a + 1, b, c)),
     [(pins.test_lgf_origin_watson, ()), (pins.test_lgf_symmetry_of_quadrature, ())]),
    ("G_L tail of the integral dropped (a constant offset)",
     lambda o: dict(lgf_quad=lambda *n: o.lgf_quad(*n) + 1e-9),
     [(pins.test_lgf_origin_watson, ())]),
    ("G_L table index with transposed components",
     lambda o: dict(table_index=lambda a, b, c: o.table_index(a, c, b) if c <= b <= a and c < b else
                    o.table_index(a, b, c)),
     [(pins.test_lgf_table_satisfies_lattice_poisson, ()), (pins.test_lgf_table_matches_pointwise_quadrature, ())]),
    ("far field: last correction term dropped",
     lambda o: dict(lgf_asym=lambda a, b, c, order=7: o.lgf_asym(a, b, c, order=max(1, order - 2))),
     [(pins.test_asymptotic_matches_quadrature, ((20, 11, 5),))]),
    ("far field: sign of the expansion", lambda o: dict(lgf_asym=lambda a, b, c, order=7: -o.lgf_asym(a, b, c, order)),
     [(pins.test_asymptotic_matches_quadrature, ((24, 0, 0),)), (pins.test_lgf_lookup_switches_to_expansion, ())]),
    ("Poisson apply scaled by dx, not dx^2",
     lambda o: dict(poisson_direct=lambda b, s, f, t, dx=1.0, R=32: o.poisson_direct(b, s, f, t, dx=np.sqrt(dx), R=R)),
     [(pins.test_poisson_direct_point_source_reproduces_table, ())]),
    ("Poisson apply with the source block read z-fastest", lambda o: dict(poisson_direct=_transposed_source(o)),
     [(pins.test_poisson_direct_point_source_reproduces_table, ()),
      (pins.test_poisson_direct_solves_lattice_poisson, ())]),
    ("E weights with I_n(alpha) for I_n(2 alpha)",
     lambda o: dict(intfactor_weights=lambda a, n: o.intfactor_weights(a / 2, n)),
     [(pins.test_intfactor_weights_are_skellam, (0.5,))]),
    ("E weights without the e^{-2 alpha} factor",
     lambda o: dict(intfactor_weights=lambda a, n: o.intfactor_weights(a, n) * np.exp(2 * a)),
     [(pins.test_intfactor_weights_are_skellam, (0.25,)), (pins.test_intfactor_semigroup, (0.1, 0.25))]),
    ("E apply for twice the time", lambda o: dict(intfactor_box=lambda a, f: o.intfactor_box(2 * a, f)),
     [(pins.test_intfactor_apply_matches_heat_equation, ())]),
    ("E apply with target block coordinates reversed",
     lambda o: dict(intfactor_blocks=lambda a, b, s, f, t: o.intfactor_blocks(a, b, s, f, np.asarray(t)[:, ::-1])),
     [(pins.test_intfactor_blocks_point_source, ())]),
    ("G_K with the sign of R(alpha) flipped",
     lambda o: dict(gk_quad=lambda a, *n: 2 * o.lgf_quad(*n) - o.gk_quad(a, *n)),
     [(pins.test_gk_laplacian_is_heat_kernel, (0.25,))]),
    ("G_K with R integrated over [0, 2 alpha]", lambda o: dict(gk_quad=lambda a, *n: o.gk_quad(2 * a, *n)),
     [(pins.test_gk_laplacian_is_heat_kernel, (0.25,)), (pins.test_gk_equals_lgf_convolved_with_heat_kernel, ())]),
    ("curl with one component's sign flipped", lambda o: dict(curl_box=_curl_with_flipped_term(o)),
     [(pins.test_curl_adjoint_pair, ()), (pins.test_mimetic_identity_of_section_2_1, ())]),
    ("curl adjoint without its minus sign", lambda o: dict(curl_adj_box=lambda w, dx=1.0: -o.curl_adj_box(w, dx)),
     [(pins.test_curl_adjoint_pair, ()), (pins.test_mimetic_identity_of_section_2_1, ())]),
    ("curl result shifted by one cell",
     lambda o: dict(curl_box=lambda u, dx=1.0: np.roll(o.curl_box(u, dx), 1, axis=-1)),
     [(pins.test_curl_adjoint_pair, ()), (pins.test_curl_orthogonality, ())]),
    ("three-point kernel with a wrong inner branch", lambda o: dict(phi3=_wrong_phi3),
     [(pins.test_phi3_moment_conditions, (0.25,))]),
    ("spreading without the 1/dx^3 of the discrete delta",
     lambda o: dict(ib_spread=lambda b, c, X, g, dx=1.0: o.ib_spread(b, c, X, g, 1.0)),
     [(pins.test_ib_interp_is_scaled_adjoint_of_spread, ())]),
    ("interpolation with marker coordinates transposed",
     lambda o: dict(ib_interp=lambda b, c, X, v: o.ib_interp(b, c, np.asarray(X)[:, ::-1], v)),
     [(pins.test_ib_interp_exact_for_linear_fields, ())]),
    ("stage: pressure correction with its sign flipped",
     lambda o: dict(stage_pc=lambda g, ds, gf, dx, R, ops: 2 * ds - o.stage_pc(g, ds, gf, dx, R, ops)),
     [(pins.test_nested_projection_satisfies_no_slip, (0.0,)),
      (pins.test_nested_projection_is_divergence_free_inside, ())]),
    ("stage: velocity correction without the regularised force",
     lambda o: dict(stage_vc=lambda g, r, dh, gf, a, dx, ops: o.stage_vc(g, r, dh, 0 * gf, a, dx, ops)),
     [(pins.test_nested_projection_satisfies_no_slip, (0.3,))]),
    ("stage: force right side without the integrating factor",
     lambda o: dict(stage_f_rhs=lambda g, r, ds, X, ub, a, dx, ops: o.stage_f_rhs(g, r, ds, X, ub, 0.0, dx, ops)),
     [(pins.test_nested_projection_satisfies_no_slip, (0.0,))]),
    ("stage: intermediate pressure with the sign of its source flipped",
     lambda o: dict(stage_ip=lambda g, r, dx, R, ops: -o.stage_ip(g, r, dx, R, ops)),
     [(pins.test_nested_projection_is_divergence_free_inside, ())]),
    ("stage: regularisation without the dx^3 of I^dagger",
     lambda o: dict(stage_regularize=lambda g, Xp, fh, dx, ops: o.stage_regularize(g, Xp, fh, dx, ops) / dx ** 3),
     [(pins.test_nested_projection_satisfies_no_slip, (0.0,))]),
]


@pytest.mark.parametrize("name,make,checks", CASES, ids=[c[0] for c in CASES])
def test_a_planted_mistake_fails_a_pin(oracle, name, make, checks):
    mutant = Mutant(oracle, **make(oracle))
    failed = []
    for fn, args in checks:
        try:
            fn(mutant, *args)
        except AssertionError:
            failed.append(fn.__name__)
    assert failed, f"no pin caught the planted mistake: {name}"
