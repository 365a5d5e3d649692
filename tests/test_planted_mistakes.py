"""Planted mistakes: every pin of the oracle must catch the slip it guards against.

Each case below alters one place of a copy of the oracle's C source -- a dropped term, a
flipped sign, a wrong index, a transposed operand, the misprint of Eq. 4 -- compiles the
copy with gcc into a temporary library, swaps it in for the real one and runs the pin
named beside it, which must then fail.  The unaltered source, compiled and swapped in the
same way, must pass every one of those pins, so a failure comes from the alteration and
not from the harness.  Nothing here touches a GPU or the CUDA library.
"""
import concurrent.futures as cf
import ctypes
import os

import pytest

import oracle
import test_oracle_pins as P

PINS = {
    "finite differences, kappa 0": lambda: P.test_kernel_derivatives_match_finite_differences(0.0),
    "finite differences, kappa 0.104": lambda: P.test_kernel_derivatives_match_finite_differences(0.104),
    "finite differences, kappa 1.3": lambda: P.test_kernel_derivatives_match_finite_differences(1.3),
    "mesh check codes": P.test_mesh_check_codes,
    "patch geometry": P.test_patch_geometry,
    "independent quadrature, distance 1": lambda: P.test_near_rule_matches_independent_quadrature(1.0),
    "independent quadrature, distance 3": lambda: P.test_near_rule_matches_independent_quadrature(3.0),
    "Gauss law over the patches": P.test_gauss_law_over_whole_patch_surface,
    "sphere row sums": P.test_sphere_row_sums_converge_to_exact_integrals,
    "near set symmetric": P.test_near_set_is_symmetric_and_contains_neighbours,
    "matvec equals assembled matrix": P.test_matvec_paths_agree_with_assembled_matrix,
    "GMRES equals dense LU": P.test_gmres_matches_dense_lu,
    "Born ion, kappa 0": lambda: P.test_born_ion_surface_solution_and_energy(0.0),
    "self term radial closed form": P.test_self_term_matches_radial_closed_form,
}

# (what the slip is, text of the oracle source, its replacement, the pin that catches it)
MISTAKES = [
    # kernels (definitions below Eq. 3)
    ("dG/dn0 with the wrong sign", "k8[2] = -n0d * G3;", "k8[2] = n0d * G3;",
     "finite differences, kappa 0.104"),
    ("Yukawa first derivative without (1 + kr)", "double g1 = (e * (1.0 + kr)) * G3;",
     "double g1 = e * G3;", "finite differences, kappa 1.3"),
    ("second derivative without its factor 3", "double G5 = 3.0 * G3 / r2;",
     "double G5 = G3 / r2;", "finite differences, kappa 0"),
    ("Yukawa second derivative without (kr)^2/3",
     "double g2 = (e * (1.0 + kr + kr * kr / 3.0)) * G5;", "double g2 = (e * (1.0 + kr)) * G5;",
     "finite differences, kappa 1.3"),
    ("screening factor exp(-kappa r^2)", "double e = exp(-kappa * r);",
     "double e = exp(-kappa * r2);", "finite differences, kappa 1.3"),
    # Eq. 6 integrands
    ("B divides the Yukawa kernel by eps_bar", "o[1] = k8[1] / ebar - k8[5];",
     "o[1] = k8[1] - k8[5] / ebar;", "independent quadrature, distance 1"),
    ("D divides only the Yukawa part by eps_bar", "o[3] = (k8[3] - k8[7]) / ebar;",
     "o[3] = k8[3] - k8[7] / ebar;", "independent quadrature, distance 1"),
    ("C takes the Laplace kernel twice", "o[2] = k8[2] - k8[6] / ebar;",
     "o[2] = k8[2] - k8[2] / ebar;", "independent quadrature, distance 1"),
    # node patch (Fig. 1)
    ("patch takes half of each triangle", "A += c->tri_area[t] / 3.0;",
     "A += c->tri_area[t] / 2.0;", "patch geometry"),
    ("patch edge midpoint on the opposite edge", "ma[k] = 0.5 * (xv[k] + xa[k]);",
     "ma[k] = 0.5 * (xa[k] + xb[k]);", "Gauss law over the patches"),
    # near rule (reading R4) and self term (reading R5)
    ("Radon weights paired with the wrong orbits",
     "double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;",
     "double w1 = (155.0 + s15) / 1200.0, w2 = (155.0 - s15) / 1200.0;",
     "independent quadrature, distance 3"),
    ("1 -> 4 split loses the middle sub-triangle",
     "        tri_quad_rec(c, x, n0, m01, m12, m20, ns, depth + 1, acc);\n", "",
     "independent quadrature, distance 1"),
    ("refinement test inverted", "dist3(x, cen) < c->refine_ratio * diam",
     "dist3(x, cen) > c->refine_ratio * diam", "independent quadrature, distance 1"),
    ("self term A with an extra 1/l", "double fa = -expm1(-x) / (fp * l);",
     "double fa = -expm1(-x) / (fp * l * l);", "self term radial closed form"),
    ("self term series without alternating signs",
     "term *= -x / jj * (double)(jj - 1) / (double)(jj - 2);",
     "term *= x / jj * (double)(jj - 1) / (double)(jj - 2);", "self term radial closed form"),
    ("self term D not divided by eps_bar", "o[3] = Dsum / c->ebar;", "o[3] = Dsum;",
     "self term radial closed form"),
    ("Gauss-Legendre weights doubled", "w[i] = 1.0 / ((1.0 - z * z) * dp * dp);",
     "w[i] = 2.0 / ((1.0 - z * z) * dp * dp);", "self term radial closed form"),
    # near set (reading R3) and far rule
    ("near test with rho_p twice", "c->c_near * (c->rho[p] + c->rho[t]);",
     "c->c_near * (c->rho[p] + c->rho[p]);", "near set symmetric"),
    ("far rule scaled by the target's area", "for (int k = 0; k < 4; k++) o[k] *= c->area[t];",
     "for (int k = 0; k < 4; k++) o[k] *= c->area[p];", "sphere row sums"),
    # Eq. 5 operator
    ("matvec adds A h", "s1 += o[1] * f[t] - o[0] * h[t];", "s1 += o[1] * f[t] + o[0] * h[t];",
     "matvec equals assembled matrix"),
    ("matvec with C and D transposed", "s2 += o[3] * f[t] - o[2] * h[t];",
     "s2 += o[2] * f[t] - o[3] * h[t];", "matvec equals assembled matrix"),
    ("second block's diagonal takes f", "double s1 = c->alpha * f[p], s2 = c->alpha * h[p];",
     "double s1 = c->alpha * f[p], s2 = c->alpha * f[p];", "matvec equals assembled matrix"),
    ("assembled C and D blocks swapped", "r2[t] = o[3]; r2[n + t] = -o[2];",
     "r2[t] = -o[2]; r2[n + t] = o[3];", "matvec equals assembled matrix"),
    ("alpha with eps_bar instead of 1/eps_bar", "c->alpha = 0.5 / c->ebar + 0.5;",
     "c->alpha = 0.5 * c->ebar + 0.5;", "Born ion, kappa 0"),
    ("eps_bar inverted", "c->ebar = eps_out / eps_in;", "c->ebar = eps_in / eps_out;",
     "Born ion, kappa 0"),
    # right-hand side (Eq. 5, reading R6)
    ("RHS normal derivative with the wrong sign",
     "s2 += q[k] * (-dot3(np, d)) / (fp * r * r * r);",
     "s2 += q[k] * dot3(np, d) / (fp * r * r * r);", "Born ion, kappa 0"),
    ("RHS second row takes G, as Eq. 4 prints it",
     "s2 += q[k] * (-dot3(np, d)) / (fp * r * r * r);", "s2 += q[k] / (fp * r);",
     "Born ion, kappa 0"),
    ("RHS first row not divided by eps_out", "*b1 = s1 / c->eps_out;", "*b1 = s1;",
     "Born ion, kappa 0"),
    # energy (reading R7)
    ("energy without eps_bar", "s += c->area[t] * (c->ebar * h[t] * G - f[t] * dGdn);",
     "s += c->area[t] * (h[t] * G - f[t] * dGdn);", "Born ion, kappa 0"),
    ("energy double layer with the wrong sign",
     "s += c->area[t] * (c->ebar * h[t] * G - f[t] * dGdn);",
     "s += c->area[t] * (c->ebar * h[t] * G + f[t] * dGdn);", "Born ion, kappa 0"),
    ("energy without 4 pi", "return E * fp * ORC_KC;", "return E * ORC_KC;",
     "Born ion, kappa 0"),
    # GMRES (Sec. 3.4, Eq. 7)
    ("Givens update of the residual with the wrong sign", "g[j + 1] = -sn[j] * g[j];",
     "g[j + 1] = sn[j] * g[j];", "GMRES equals dense LU"),
    ("Givens rotation with the wrong sign", "H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;",
     "H[(i + 1) * m + j] = sn[i] * a + cs[i] * bb;", "GMRES equals dense LU"),
    ("back substitution with H transposed", "s -= H[i * m + k] * yv[k];",
     "s -= H[k * m + i] * yv[k];", "GMRES equals dense LU"),
    ("Gram-Schmidt skips the first basis vector",
     "for (int i = 0; i <= j; i++) {\n                double hij = vdot(n2, w, V + (size_t)i * n2); inner++;\n"
     "                H[i * m + j] = hij;",
     "for (int i = 1; i <= j; i++) {\n                double hij = vdot(n2, w, V + (size_t)i * n2); inner++;\n"
     "                H[i * m + j] = hij;", "GMRES equals dense LU"),
    # mesh checks (closed, manifold, outward)
    ("mesh check accepts inward orientation", "if (vol <= 0) return 4;",
     "if (vol < -1e300) return 4;", "mesh check codes"),
    ("mesh check accepts unmatched edges", "if (dir[i] != rev[i]) { bad = 1; break; }", "",
     "mesh check codes"),
]


@pytest.fixture(scope="module")
def libraries(tmp_path_factory):
    """The unaltered source and one altered copy per mistake, compiled in parallel."""
    src = open(oracle._SRC).read()
    d = tmp_path_factory.mktemp("planted")
    jobs = [(str(d / "clean.c"), src)]
    for i, (what, old, new, _) in enumerate(MISTAKES):
        assert src.count(old) == 1, "the oracle source no longer holds the text for: " + what
        jobs.append((str(d / ("m%02d.c" % i)), src.replace(old, new)))
    for path, text in jobs:
        with open(path, "w") as fh:
            fh.write(text)
    with cf.ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        libs = list(ex.map(lambda j: oracle.compile_source(j[0], j[0][:-2] + ".so"), jobs))
    return libs[0], libs[1:]


def _run_with(lib_path, pin):
    """Run one pin with the oracle library at lib_path in place of the real one."""
    real = oracle._load()
    oracle._lib = oracle.configure(ctypes.CDLL(lib_path))
    try:
        PINS[pin]()
    finally:
        oracle._lib = real


def test_unaltered_copy_passes_every_pin(libraries):
    clean, _ = libraries
    for pin in sorted({m[3] for m in MISTAKES}):
        _run_with(clean, pin)


@pytest.mark.parametrize("k", range(len(MISTAKES)), ids=[m[0] for m in MISTAKES])
def test_planted_mistake_is_caught(libraries, k):
    _, altered = libraries
    what, _, _, pin = MISTAKES[k]
    with pytest.raises(AssertionError):
        _run_with(altered[k], pin)
