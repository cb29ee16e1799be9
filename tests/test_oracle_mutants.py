"""The pins of test_oracle_pins.py must catch plausible mistakes in the oracle.

Each case copies oracle.c, plants one mistake (on the CPU; nothing here touches a GPU),
builds the copy, and runs the pin suite against it in a subprocess: the suite must fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "tf weight swapped": ("e->rgba[c] = (1.0 - w) * a + w * b;", "e->rgba[c] = w * a + (1.0 - w) * b;"),
    "first sample floor": ("*k0 = (int64_t)ceil(a) + s->dk0;", "*k0 = (int64_t)floor(a) + s->dk0;"),
    "last sample inclusive": ("*k1 = (int64_t)ceil(b) + s->dk1;", "*k1 = (int64_t)ceil(b) + 1 + s->dk1;"),
    "colour without transmittance": ("for (int c = 0; c < 3; ++c) C[c] += T * a * e.rgba[c];",
                                     "for (int c = 0; c < 3; ++c) C[c] += a * e.rgba[c];"),
    "voxel centre offset dropped": ("double q = p[a] - 0.5;", "double q = p[a];"),
    "axes swapped in the index": ("int64_t li = (z * s->ny + y) * s->nx + x;",
                                  "int64_t li = (y * s->nz + z) * s->nx + x;"),
    "termination before the crossing sample": (
        "        if (ert_on && 1.0 - T >= s->ert) break;",
        "        if (ert_on && 1.0 - T * (1.0 - a) >= s->ert) break;"),
    "termination window widened 100x": ("fabs((1.0 - T) - s->ert) <= 2.0 * E + ert_win",
                                         "fabs((1.0 - T) - s->ert) <= 200.0 * E + 100.0 * ert_win"),
    "termination flag dropped": ("if (ert_on && fabs((1.0 - T) - s->ert) <= 2.0 * E + ert_win) r->flags |= FLAG_ERT;",
                                 ""),
    "termination window ignores the position error": ("*dv = s->pos_err * sumD + U32 * (sumD + 3.0 * M);",
                                                      "*dv = U32 * (sumD + 3.0 * M);"),
    "end-sample window widened 100x": ("return ldexp(1.0, -36) * (fabs(o[a]) + n[a] + fabs(t)) / (fabs(d[a]) * s->step);",
                                       "return ldexp(100.0, -36) * (fabs(o[a]) + n[a] + fabs(t)) / (fabs(d[a]) * s->step);"),
    "first-sample flag dropped": ("if (an >= 0 && tn > 0.0 && frac_dist(a) <= end_window(s, o, d, an, tn)) *flags |= FLAG_K0;",
                                  ""),
    "last-sample flag dropped": ("if (af >= 0 && frac_dist(b) <= end_window(s, o, d, af, tf)) *flags |= FLAG_K1;", ""),
    "termination variant not shifted": ("nstop = r0.nsamp + s->dstop;", "nstop = r0.nsamp;"),
    "adjoint node alternative dropped": ("    if (fabs(x - j) > xr || j < 0.0 || j > (double)(s->ntf - 1)) return 0.0;",
                                         "    return 0.0;"),
    "adjoint flagged rays not bounded": ("    if (!rr.flags) return;", "    return;"),
    "perspective direction not normalised": ("for (int a = 0; a < 3; ++a) d[a] = dd[a] / len;",
                                             "for (int a = 0; a < 3; ++a) d[a] = dd[a];"),
    "pixel corner instead of centre": ("double u = l + ((double)px + 0.5) * (r - l) / (double)c->width;",
                                       "double u = l + ((double)px) * (r - l) / (double)c->width;"),
    "adjoint suffix sign": ("ga += g[c] * q->T * (q->rgb[c] - R[c]);", "ga += g[c] * q->T * (q->rgb[c] + R[c]);"),
    "adjoint tf weight swapped": ("dtf[4 * q->e.i + c] += (1.0 - q->e.w) * gch[c];",
                                  "dtf[4 * q->e.i + c] += q->e.w * gch[c];"),
    "mip keeps the minimum": ("            if (v > m) m = v;\n            continue;", "            if (!(v > m) || m == -INFINITY) m = v;\n            continue;"),
    "slab starts behind the eye": [("double lo = 0.0, hi = INFINITY;", "double lo = -INFINITY, hi = INFINITY;"),
                                   ("    if (*k0 < 0) *k0 = 0;\n", "")],
    "slab exit takes the farther plane": ("        if (th < hi) {", "        if (th > hi || hi == INFINITY) {"),
    "sort-last folds back to front": ("if (x->key != y->key) return x->key < y->key ? -1 : 1;",
                                      "if (x->key != y->key) return x->key < y->key ? 1 : -1;"),
    "sort-last orthographic key sign": ("q->key += d[a] > 0 ? b[a] : (d[a] < 0 ? -b[a] : 0);",
                                        "q->key += d[a] > 0 ? -b[a] : (d[a] < 0 ? b[a] : 0);"),
    "sort-last perspective key unsigned distance": (
        "q->key += b[a] > e[a] ? b[a] - e[a] : e[a] - b[a];", "q->key += b[a] - e[a];"),
    "touch marks half the corners": ("for (int c = 0; c < 8; ++c) __atomic_store_n",
                                     "for (int c = 0; c < 4; ++c) __atomic_store_n"),
    "bf16 truncates": ("u = (u + 0x7fffu + lsb) & 0xffff0000u;", "u = u & 0xffff0000u;"),
    "bf16 ties away from zero": ("u = (u + 0x7fffu + lsb) & 0xffff0000u;", "u = (u + 0x8000u) & 0xffff0000u;"),
    "mip adjoint tf weight swapped": ("dtf[4 * e->i + c] += (1.0 - e->w) * g[c];", "dtf[4 * e->i + c] += e->w * g[c];"),
    "adjoint suffix transmittance kept at one": ("        P *= (1.0 - q->a);\n", ""),
    "adjoint colour gradient without opacity": ("gc[c] = g[c] * q->T * q->a;", "gc[c] = g[c] * q->T;"),
    "tf slope where the lookup is clamped": (
        "e->slope[c] = inside ? (b - a) * (double)(s->ntf - 1) / (s->vmax - s->vmin) : 0.0;",
        "e->slope[c] = (b - a) * (double)(s->ntf - 1) / (s->vmax - s->vmin);"),
    "pyramid divides by four at edges": ("cur[4 * (y * lw + x) + c] = acc[c] / (double)n;",
                                         "cur[4 * (y * lw + x) + c] = acc[c] / 4.0;"),
    "pyramid tiles transposed": ("return ((y / tile) * tx + x / tile) * tile * tile + (y % tile) * tile + (x % tile);",
                                 "return ((x / tile) * tx + y / tile) * tile * tile + (y % tile) * tile + (x % tile);"),
    "overlay without the pixel-centre offset": ("double X0 = (u0 - l) * sx - 0.5, Y0 = (t - v0) * sy - 0.5;",
                                                 "double X0 = (u0 - l) * sx, Y0 = (t - v0) * sy - 0.5;"),
    "overlay keeps the first box": ("if (key[py * W + px] < k) key[py * W + px] = k;",
                                    "if (key[py * W + px] == 0) key[py * W + px] = k;"),
    "overlay blend without transmittance": (
        "img[4 * i + ch] = a * (double)c[ch] + (1.0 - a) * img[4 * i + ch];",
        "img[4 * i + ch] = a * (double)c[ch] + img[4 * i + ch];"),
    "overlay perspective without the divide": ("u0 = c0[0] / c0[2];", "u0 = c0[0];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    sites = MUTANTS[name]
    text = open(SRC).read()
    for old, new in (sites if isinstance(sites, list) else [sites]):
        assert text.count(old) == 1, f"mutation site not found once: {name}"
        text = text.replace(old, new)
    src = tmp_path / "oracle_mutant.c"
    src.write_text(text)
    lib = tmp_path / "oracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=gnu11", "-ffp-contract=off",
                           str(src), "-o", str(lib), "-lm"])
    env = dict(os.environ, VR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"the pins did not catch: {name}\n{r.stdout[-2000:]}"
