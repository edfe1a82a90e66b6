"""The pins must catch plausible mistakes in the oracle.

Each case compiles a copy of the oracle with one planted mistake (a dropped
term, a wrong sign, a transposed index ...) and runs the pin module expected to
catch it against that copy; the module must fail.  CPU only.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rt_oracle.cpp")

MUTATIONS = {
    # continuous absorption without the (1 - albedo) factor
    "absorption_albedo": ("T dep = T(1.0 - alb) * L", "T dep = T(1.0) * L", "test_oracle_transport.py"),
    # peel-off phase function evaluated at the wrong cosine sign
    "peel_phase_sign": ("hg_phase(P.g[lam], k.x * f.kobs.x + k.y * f.kobs.y + k.z * f.kobs.z)",
                        "hg_phase(P.g[lam], -(k.x * f.kobs.x + k.y * f.kobs.y + k.z * f.kobs.z))",
                        "test_oracle_transport.py"),
    # interaction drawn without forcing (plain exponential optical depth)
    "unforced": ("const T tau_star = -log1p(-T(u[0]) * one_minus_E);", "const T tau_star = -log1p(-T(u[0]));",
                 "test_oracle_transport.py"),
    # pixel index transposed
    "pixel_transpose": ("int64_t pix = (int64_t)iy * f.nx + (int64_t)ix;\n        tally",
                        "int64_t pix = (int64_t)ix * f.nx + (int64_t)iy;\n        tally", "test_oracle_transport.py"),
    # deposit into the next cell along the path
    "absorption_index": ("tally.absorb(lam, segs[i].cell, dep);",
                         "tally.absorb(lam, segs[i + 1 < segs.size() ? i + 1 : i].cell, dep);",
                         "test_oracle_transport.py"),
    # Philox round uses the wrong product half
    "philox_half": ("uint32_t n0 = hi1 ^ c[1] ^ k0;", "uint32_t n0 = hi0 ^ c[1] ^ k0;", "test_oracle_rng.py"),
    # walk always steps towards +axis
    "walk_direction": ("idx[axis] += comp(k, axis) > 0 ? 1 : -1;", "idx[axis] += 1;", "test_oracle_geometry.py"),
    # azimuth drawn over half a turn
    "half_azimuth": ("return rotate_dir(k, hg_sample(g, u1), 2.0 * M_PI * u2);",
                     "return rotate_dir(k, hg_sample(g, u1), M_PI * u2);", "test_oracle_optics.py"),
    # scattering directions drawn with the opposite asymmetry (forward and
    # backward scattering swapped after the first event)
    "scatter_g_sign": ("return rotate_dir(k, hg_sample(g, u1), 2.0 * M_PI * u2);",
                       "return rotate_dir(k, hg_sample(-g, u1), 2.0 * M_PI * u2);", "test_oracle_analog.py"),
    # rounding fallback of the inversion placed at the end of the path instead
    # of the end of the last dusty segment
    "fallback_last_segment": ("for (size_t i = 0; i < segs.size(); ++i) if (val(tau[i + 1]) > val(tau[i])) hit = i;",
                              "hit = segs.size() - 1;", "test_oracle_interaction.py"),
    # interaction point left where rounding put it (no move into its cell)
    "no_cell_clamp": ("      set_comp(x, a, xa);\n    }\n    if (clamped)", "    }\n    if (clamped)",
                      "test_oracle_interaction.py"),
    # inversion remainder measured from the segment's far end
    "inversion_remainder": ("(tau_star - tau[hit]) / (T(kap)", "(tau_star - tau[hit + 1]) / (T(kap)",
                            "test_oracle_interaction.py"),
    # SED instrument recording scattered light as direct
    "sed_channel": ("if (f.channels == 3) tally.pixel((int)q, scattered ? 2 : 1, lam, 0, value, pid, event);",
                    "if (f.channels == 3) tally.pixel((int)q, 1, lam, 0, value, pid, event);", "test_oracle_sed.py"),
    # rectilinear grid planes read one edge off
    "rect_plane_index": ("return kind == 2 ? edges[axis][(size_t)i] :",
                         "return kind == 2 ? edges[axis][(size_t)(i > 0 ? i - 1 : 0)] :", "test_oracle_rectilinear.py"),
    # Planck function with the wrong power of the wavelength
    "planck_power": ("return 1.0 / (std::pow(lambda_um, 5.0) * std::expm1(kC2 / (lambda_um * T)));",
                     "return 1.0 / (std::pow(lambda_um, 4.0) * std::expm1(kC2 / (lambda_um * T)));",
                     "test_oracle_panchromatic.py"),
    # dust emission from the extinction instead of the absorption coefficient
    "emission_albedo": ("scale * P.kappa[(size_t)l] * (1.0 - P.albedo[(size_t)l]) * w[(size_t)l]",
                        "scale * P.kappa[(size_t)l] * w[(size_t)l]", "test_oracle_panchromatic.py"),
    # emitting cell drawn uniformly instead of by luminosity
    "dust_cell_uniform": ("const int64_t cell = std::min<int64_t>(c, (int64_t)cum.size() - 1);",
                          "const int64_t cell = std::min<int64_t>((int64_t)(u[0] * cum.size()), (int64_t)cum.size() - 1); (void)c;",
                          "test_oracle_panchromatic.py"),
    # k-d tree children taken in the wrong order
    "bintree_child_order": ("node = child[node] + (upper ? 1 : 0);", "node = child[node] + (upper ? 0 : 1);",
                            "test_oracle_bintree.py"),
    # Voronoi walk ignoring the last face of every cell
    "voronoi_last_face": ("for (int64_t f = G.offsets[cell]; f < G.offsets[cell + 1]; ++f) {",
                          "for (int64_t f = G.offsets[cell]; f + 1 < G.offsets[cell + 1]; ++f) {",
                          "test_oracle_voronoi.py"),
    # Voronoi bisecting plane through the cell's own site instead of the midpoint
    "voronoi_plane_offset": ("(T(0.5 * (sc[0] + sj[0])) - x.x)", "(T(sc[0]) - x.x)", "test_oracle_voronoi.py"),
    # derivative of exp with the wrong sign
    "dual_exp_sign": ("inline Dual exp(Dual a) { double e = std::exp(a.v); return {e, e * a.d}; }",
                      "inline Dual exp(Dual a) { double e = std::exp(a.v); return {e, -e * a.d}; }",
                      "test_oracle_transport.py"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new, module = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    cpp = tmp_path / f"{name}.cpp"
    so = tmp_path / f"{name}.so"
    cpp.write_text(src.replace(old, new, 1))
    subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                    str(cpp), "-o", str(so)], check=True)
    env = dict(os.environ, RT_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", module)], env=env, capture_output=True, text=True, cwd=ROOT)
    assert r.returncode == 1, f"mutation {name} was not caught:\n{r.stdout[-2000:]}"
