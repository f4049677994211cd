"""Mutation check of the oracle's pins (a tool, not collected by pytest).

Plants one deliberate one-line mistake at a time in a copy of oracle/oracle.c,
builds it, and runs the CPU tests against that build (ORACLE_LIB points the
oracle wrapper at it). Every mutant must make some test fail: a mutant that
passes would be a mistake the pins cannot see.

    python tests/oracle_mutations.py            # all mutants
    python tests/oracle_mutations.py tie_id     # some of them

Builds go to oracle/_mutants/ (git-ignored) and are removed afterwards.
"""
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
WORK = os.path.join(ROOT, "oracle", "_mutants")

# name: (text in oracle.c, replacement)
MUTANTS = {
    "philox_nobump": ("k0 += PHILOX_W0;", "k0 += 0;"),
    "uniform_shift": ("(x[0] >> 8)", "(x[0] >> 9)"),
    "onb_sign": ("b2[2] = -n[1];", "b2[2] = n[1];"),
    "cos_z": ("z = sqrt(1.0 - u1)", "z = sqrt(u1)"),
    "sphere_far": ("if (t0 > tmin && t0 <= tmax) { *t_out = t0; return 1; }", ""),
    "cyl_noclip": ("if (!hit && s >= 0.0 && s <= L)", "if (!hit)"),
    "cyl_dp": ("double tc = -dot3(wp, dp) / A;", "double tc = dot3(wp, dp) / A;"),
    "dda_tie": ("if (nr->id1 != OR_MISS && nr->t1 <= dda_cell_exit(&w)) break;",
                "if (nr->id1 != OR_MISS) break;"),
    "anyhit_nocount": ("        cnt->cells++;\n        int64_t c = ((int64_t)w.c[2] * gr->n[1] + w.c[1]) * gr->n[0] + w.c[0];\n"
                       "        for (int64_t i = gr->start[c]; i < gr->start[c + 1]; ++i) {",
                       "        int64_t c = ((int64_t)w.c[2] * gr->n[1] + w.c[1]) * gr->n[0] + w.c[0];\n"
                       "        for (int64_t i = gr->start[c]; i < gr->start[c + 1]; ++i) {"),
    "anyhit_kind": ("            if (id < sc->S) cnt->sph++; else cnt->cyl++;", "            cnt->sph++;"),
    "anyhit_one_cell": ("    } while (dda_next(gr, &w));\n    return 0;", "    } while (0);\n    return 0;"),
    "grid_nopad": ("c0[k] = cell_coord(gr, k, a[k] - pad); c1[k] = cell_coord(gr, k, b[k] + pad);",
                   "c0[k] = cell_coord(gr, k, a[k] + 0.3); c1[k] = cell_coord(gr, k, b[k] - 0.3);"),
    "refine_normal": ("if (dot3(n, d) > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }",
                      "if (dot3(n, d) < 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }"),
    "shade_refl": ("double r[3] = {2.0 * ndl * n[0] - L[0]", "double r[3] = {2.0 * ndl * n[0] + L[0]"),
    "shade_scale": ("diff += sp[0] * lI[l] * sp[3] * ndl;", "diff += lI[l] * sp[3] * ndl;"),
    "ray_row": ("double v = cam[14] * (1.0 - 2.0 * y / H);", "double v = cam[14] * (2.0 * y / H - 1.0);"),
    "ray_halfpix": ("(double)i + (a + 0.5) / m", "(double)i + (a + 0.0) / m"),
    "aa_subrow": ("(double)j + (b + 0.5) / m", "(double)j + (a + 0.5) / m"),
    "aa_counter": ("oracle_ao_uniforms(qf, (uint32_t)s", "oracle_ao_uniforms((uint32_t)q, (uint32_t)s"),
    "aa_mean": ("const double mm = (double)m * m;", "const double mm = (double)m;"),
    "aa_layout": ("const int64_t sub = k * m * m + b * m + a;", "const int64_t sub = k * m * m + a * m + b;"),
    "ao_eps": ("double ao_o[3] = {p[0] + sp[6] * n[0]", "double ao_o[3] = {p[0] - sp[6] * n[0]"),
    "tie_id": ("if (t < nr->t1 || (t == nr->t1 && uid < nr->id1))",
               "if (t < nr->t1 || (t == nr->t1 && uid > nr->id1))"),
    "aabb_cyl": ("double e = c[6] * sqrt(fmax(0.0, 1.0 - ak * ak));", "double e = 0.0;"),
    "shadow_inv": ("lit[l] = !world_anyhit(&w, ao_o, ldir + 3 * l, INFINITY, &sc_);",
                   "lit[l] = world_anyhit(&w, ao_o, ldir + 3 * l, INFINITY, &sc_);"),
    "shadow_flag": ("if (sp[11] != 0.0 && dot3(n, ldir + 3 * l) > 0.0)",
                    "if (sp[11] == 0.0 && dot3(n, ldir + 3 * l) > 0.0)"),
    # the grazing classifier (which pixels hit-id parity is asserted on)
    "graze_disc_big": ("#define GRAZE_DISC 1e-4", "#define GRAZE_DISC 1e-3"),
    "graze_disc_small": ("#define GRAZE_DISC 1e-4", "#define GRAZE_DISC 1e-5"),
    "graze_tie_big": ("#define GRAZE_TIE 1e-5", "#define GRAZE_TIE 1e-4"),
    "graze_tie_small": ("#define GRAZE_TIE 1e-5", "#define GRAZE_TIE 1e-6"),
    "graze_end_big": ("#define GRAZE_END 1e-4", "#define GRAZE_END 1e-3"),
    "graze_tclose_sign": ("        g->t_close = -b;", "        g->t_close = b;"),
    "graze_miss": ("if (nr->id1 == OR_MISS) return nr->t_graze < INFINITY;",
                   "if (nr->id1 == OR_MISS) return 0;"),
    "graze_before": ("if (nr->t_graze <= nr->t1 * (1.0 + GRAZE_TIE) + 1e-9) return 1;",
                     "if (nr->t_graze < INFINITY) return 1;"),
    "graze_tmin": ("fabs(g.disc_rel) < GRAZE_DISC && g.t_close > tmin &&", "fabs(g.disc_rel) < GRAZE_DISC &&"),
    "graze_near_root": ("    if (g) g->t_near = t0;", ""),
    "graze_far_root_end": ("        for (int k = 0; k < 2; ++k) {\n            if (g.end_mrg[k]",
                           "        for (int k = 1; k < 2; ++k) {\n            if (g.end_mrg[k]"),
    "graze_tube_segment": ("&& g.s_out <= GRAZE_END * (L + 1.0) &&", "&&"),
    "graze_runner_up": ("    nr->id2 = b.id2;", "    nr->id2 = b.id1;"),
    "graze_object": ("        nr->id_graze = (uint32_t)id;\n    }\n    if (id >= sc->S) {",
                     "        nr->id_graze = OR_MISS;\n    }\n    if (id >= sc->S) {"),
}


def run(names):
    src = open(SRC).read()
    os.makedirs(WORK, exist_ok=True)
    missed = []
    try:
        for name in names:
            old, new = MUTANTS[name]
            # (a line the count and the scatter pass share is mutated in both)
            assert src.count(old) >= 1, f"{name}: the text to mutate is not in oracle.c"
            d = os.path.join(WORK, name)
            os.makedirs(d, exist_ok=True)
            c_file, so_file = os.path.join(d, "oracle.c"), os.path.join(d, "liboracle.so")
            open(c_file, "w").write(src.replace(old, new))
            # the oracle's own build flags (oracle/build.py)
            r = subprocess.run([os.environ.get("CC", "gcc"), "-fopenmp", "-O2", "-std=c11", "-D_GNU_SOURCE",
                                "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off", c_file, "-o", so_file,
                                "-lm"], capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"{name}: build failed\n{r.stderr}")
            env = dict(os.environ, ORACLE_LIB=so_file)
            r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests"), "-q", "-x",
                                "-m", "not gpu", "-p", "no:cacheprovider"], env=env, capture_output=True,
                               text=True, cwd=ROOT)
            caught = r.returncode != 0
            last = (r.stdout.strip().splitlines() or [""])[-1]
            print(f"{name:16s} caught={caught}  {last}", flush=True)
            if not caught:
                missed.append(name)
    finally:
        shutil.rmtree(WORK, ignore_errors=True)
    return missed


if __name__ == "__main__":
    sel = sys.argv[1:] or list(MUTANTS)
    missed = run(sel)
    print("all caught" if not missed else f"NOT caught: {missed}")
    sys.exit(1 if missed else 0)
