"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of ``oracle/vi_oracle.c`` (a dropped
term, a wrong sign or index, a transposed operand, an off-by-one), builds it on
the CPU and runs the pin suite against it; the suite has to fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vi_oracle.c")

MUTATIONS = {
    "inclusive-buffer": ("double stored = s->T[t];", "double stored = s->T[t] * (1.0 - alpha);"),
    "slice-off-by-one": ("fmaf((float)k, lt->dL, lt->min)", "fmaf((float)(k + 1), lt->dL, lt->min)"),
    "slice-floor-not-nearest": ("float lh = lam + 0.5f;", "float lh = lam;"),
    "voxel-corner-not-centre": ("float x = fmaf(P[a], (float)N[a], -0.5f);",
                                "float x = fmaf(P[a], (float)N[a], 0.0f);"),
    "trilinear-weight-swap": ("double w = (bx ? f[0] : 1.0 - f[0]) * (by ? f[1] : 1.0 - f[1]) * (bz ? f[2] : 1.0 - f[2]);\n        acc += w * voxel(v, bx ? hi[0] : lo[0], by ? hi[1] : lo[1], bz ? hi[2] : lo[2]);\n    }\n    return acc;\n}\n\n/* Same",
                              "double w = (bx ? 1.0 - f[0] : f[0]) * (by ? f[1] : 1.0 - f[1]) * (bz ? f[2] : 1.0 - f[2]);\n        acc += w * voxel(v, bx ? hi[0] : lo[0], by ? hi[1] : lo[1], bz ? hi[2] : lo[2]);\n    }\n    return acc;\n}\n\n/* Same"),
    "tf-scale-M": ("* (double)(tf->M - 1);", "* (double)(tf->M);"),
    "back-to-front": ("C[ch] = C[ch] + (1.0 - A) * csrc;", "C[ch] = (1.0 - alpha) * C[ch] + csrc;"),
    "u-v-transposed": ("ray->lo[1] = fmaf(dot3f(oc, lt->U)", "ray->lo[1] = fmaf(dot3f(oc, lt->V)"),
    "light-sign": ("o->L[a] = dir[a] / len;", "o->L[a] = -dir[a] / len;"),
    "cone-away-from-light": ("o[0] = -(float)ring;", "o[0] = (float)ring;"),
    "cone-rotation-sign": ("case 1: *cu = -bv; *cv = bu; break;", "case 1: *cu = bv; *cv = bu; break;"),
    "cone-radius-dropped-tan": ("float radw = dist * tanphi;", "float radw = dist;"),
    "shell-radius-units": ("float r = ((float)q * ro->shell_radius_vox) / (float)fr->Nmax;",
                           "float r = ((float)q * ro->shell_radius_vox) / (float)(2 * fr->Nmax);"),
    "shells-same-radius": ("float r = ((float)q * ro->shell_radius_vox) / (float)fr->Nmax;",
                           "float r = ro->shell_radius_vox / (float)fr->Nmax;"),
    "depth-extinction-sign": ("double D = s->T[t] + (-log1p(-alpha));",
                              "double D = s->T[t] + log1p(alpha);"),
    "depth-cap-lower": ("#define ORC_DEPTH_MAX 64.0", "#define ORC_DEPTH_MAX 16.0"),
    "depth-exp-sign": ("return ro->quantity == ORC_OPTICAL_DEPTH ? exp(-v) : v;",
                       "return ro->quantity == ORC_OPTICAL_DEPTH ? exp(v) : v;"),
    "depth-comp-n-sign": ("stored = stored - (double)s->opt->comp_n * log1p(alpha);",
                          "stored = stored + (double)s->opt->comp_n * log1p(alpha);"),
    "slice-lerp-weights-swapped": ("v = (1.0 - w) * b0 + w * b1;", "v = w * b0 + (1.0 - w) * b1;"),
    "point-axis-away-from-centre": ("float q[3] = {0.5f - pos[0], 0.5f - pos[1], 0.5f - pos[2]};",
                                    "float q[3] = {pos[0] - 0.5f, pos[1] - 0.5f, pos[2] - 0.5f};"),
    "point-half-angle-sine": ("o->h = hs / sqrtf(dc2 - hs2);", "o->h = hs / sqrtf(dc2);"),
    "point-depth-not-from-light": ("float d = dot3f(o->L, V) - pa;", "float d = dot3f(o->L, V);"),
    "point-no-perspective-divide": ("float su = dot3f(e, lt->U) / ds;", "float su = dot3f(e, lt->U);"),
    "point-parallel-columns": ("P[a] = fmaf(sk, w, lt->P[a]);",
                               "P[a] = fmaf(sk, lt->L[a], fmaf(v, lt->V[a], fmaf(u, lt->U[a], lt->P[a]))) + 0.0f * w;"),
    "point-cone-away-from-light": ("for (int a = 0; a < 3; ++a) c[a] = fmaf(-dist, w[a], S[a]);",
                                   "for (int a = 0; a < 3; ++a) c[a] = fmaf(dist, w[a], S[a]);"),
    "point-cone-turn-sign": ("cross3f(w, B[0], B[1]);", "cross3f(B[0], w, B[1]);"),
    "point-shell-radius": ("o[a] = sgn ? S[a] - r : S[a] + r;", "o[a] = sgn ? S[a] - r : S[a] + 2.0f * r;"),
    "slice-lerp-nearest-base": ("int k0 = floor_clamp(lam, 0, lt->n - 1);",
                                "int k0 = floor_clamp(lam + 0.5f, 0, lt->n - 1);"),
    "sample-count-le": ("if (!(t < ray.t1)) break;", "if (!(t <= ray.t1)) break;"),
    "opacity-correction-exponent": ("alpha = 1.0 - pow(1.0 - alpha, s->spacing_vox * column_stretch(s->lt, i, (int)j));",
                                    "alpha = 1.0 - pow(1.0 - alpha, 1.0 / (s->spacing_vox * column_stretch(s->lt, i, (int)j)));"),
    "background-not-weighted": ("o[ch] = outC[ch] + (1.0 - outA) * (double)ro->bg[ch];",
                                "o[ch] = outC[ch] + (double)ro->bg[ch];"),
    "emission-not-opacity-weighted": ("double csrc = lf * (double)ro->color[ch] * alpha * rgba[ch];",
                                      "double csrc = lf * (double)ro->color[ch] * rgba[ch];"),
    "light-colour-dropped": ("double csrc = lf * (double)ro->color[ch] * alpha * rgba[ch];",
                             "double csrc = lf * alpha * rgba[ch];"),
    "eq8-max-as-min": ("float d = dot3f(o->L, V);\n        if (c == 0 || d < mn) mn = d;\n        if (c == 0 || d > mx) mx = d;",
                       "float d = dot3f(o->L, V);\n        if (c == 0 || d < mn) mn = d;\n        if (c == 0 || d < mx) mx = d;"),
    "basis-axis-most-aligned": ("if (fabsf(o->L[1]) < fabsf(o->L[ax])) ax = 1;",
                                "if (fabsf(o->L[1]) > fabsf(o->L[ax])) ax = 1;"),
    "ert-threshold-shifted": ("const double ert = (double)ro->ert, band = ro->ert_band;",
                              "const double ert = (double)ro->ert + 0.03, band = ro->ert_band;"),
    "ert-window-start-at-threshold": ("if (lo_at < 0 && A > ert - band) {",
                                      "if (lo_at < 0 && A > ert) {"),
    "ert-band-on-wrong-side": ("if (A > ert + band) break;", "if (A > ert - band) break;"),
    "ert-outcount-from-window-end": ("        outcount = Mcount;\n", "        outcount = count;\n"),
    "ert-alt-one-sample-late": ("""            if (lo_at < 0 && A > ert - band) {
                lo_at = (long long)i;
                LC[0] = C[0]; LC[1] = C[1]; LC[2] = C[2]; LA = A; Lcount = count;
            }""", """            if (lo_at >= 0 && Lcount == 0) {
                LC[0] = C[0]; LC[1] = C[1]; LC[2] = C[2]; LA = A; Lcount = count;
            }
            if (lo_at < 0 && A > ert - band) lo_at = (long long)i;"""),
    "ert-alt-always-window-end": ("if (main_at != lo_at) {", "if (0) {"),
    "ert-wide-window-off-by-one": ("amb = last - lo_at >= 2 ? 2 : 1;", "amb = last - lo_at >= 1 ? 2 : 1;"),
    "comp-n-inverted": ("stored = stored * pow(1.0 + alpha, (double)s->opt->comp_n);",
                        "stored = stored / pow(1.0 + alpha, (double)s->opt->comp_n);"),
    "texel-centre-offset": ("float sk, float P[3]) {\n    float qi = (float)(2 * i + 1) / (float)lt->R;",
                            "float sk, float P[3]) {\n    float qi = (float)(2 * i) / (float)lt->R;"),
    "shadow-at-sample-light-coords-dropped-kappa": ("ray->ld[0] = dot3f(lt->L, ray->d) * lt->kappa;",
                                                    "ray->ld[0] = dot3f(lt->L, ray->d);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mutated = tmp_path / "vi_oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libvi_oracle_mut.so"
    subprocess.run([os.environ.get("CC", "cc"), "-std=c11", "-O2", "-ffp-contract=off",
                    "-fno-fast-math", "-fPIC", "-shared", "-pthread", "-o", str(so),
                    str(mutated), "-lm"], check=True)
    env = dict(os.environ, VI_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutation {name}:\n{r.stdout[-2000:]}"
