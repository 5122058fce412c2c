"""Planted mistakes in the oracle, each caught by its pins.

Each case copies oracle/pic_oracle.c, replaces one snippet of it (a wrong
sign, factor, index or constant, a dropped term, a step taken a step late),
compiles the copy with the oracle's own flags and runs the listed pin tests
of tests/test_oracle_*.py against it: at least one of them must fail.  The
unplanted oracle passes the same pins in those files.  This is the check
that the pins constrain every routine of the oracle, not only its shape."""
import importlib.util
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
TESTS = os.path.dirname(os.path.abspath(__file__))

# (what the mistake is, the text in pic_oracle.c, its replacement,
#  the pins that must catch it: (file, test function, parameters))
CASES = [
    ("SplitMix64: first xor-shift by 31 instead of 30",
     "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;",
     [("test_oracle_basics", "test_splitmix64_published_vector", {})]),
    ("linear shape: 1 - d^2 instead of 1 - |d|",
     "return a < 1.0 ? 1.0 - a : 0.0;", "return a < 1.0 ? 1.0 - a * a : 0.0;",
     [("test_oracle_basics", "test_shape_partition_of_unity_and_moments", {"order": 1})]),
    ("quadratic shape: centre piece 3/4 - d^2/2",
     "return 0.75 - a * a;", "return 0.75 - 0.5 * a * a;",
     [("test_oracle_basics", "test_shape_partition_of_unity_and_moments", {"order": 2})]),
    ("density profile: cos(2 m pi zeta)",
     "cos((double)m * PI_ * zeta)", "cos((double)m * TWO_PI * zeta)",
     [("test_oracle_basics", "test_density_profile", {})]),
    ("gather: Ex at integer x",
     "{0.5, 0.0, 0.0}, /* Ex (i+1/2, j,     k    ) */", "{0.0, 0.0, 0.0}, /* Ex */",
     [("test_oracle_basics", "test_gather_reproduces_linear_fields", {"dim": 2, "order": 1})]),
    ("gather: support starting one node too low (the top node of the quadratic shape lost)",
     "const int64_t bx = (int64_t)floor(xi) - 1, bz = (int64_t)floor(zi) - 1;\n    const int zmax",
     "const int64_t bx = (int64_t)floor(xi) - 2, bz = (int64_t)floor(zi) - 1;\n    const int zmax",
     [("test_oracle_basics", "test_gather_reproduces_linear_fields", {"dim": 2, "order": 2})]),
    ("Boris: full instead of half electric impulse",
     "const double eps = PI_ * q_over_m * dt;", "const double eps = TWO_PI * q_over_m * dt;",
     [("test_oracle_particles", "test_boris_uniform_e", {}),
      ("test_oracle_particles", "test_boris_uniform_b_rotation", {})]),
    ("Boris: sign of one component of u- x t",
     "up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);", "up[0] = um[0] - (um[1] * t[2] - um[2] * t[1]);",
     [("test_oracle_particles", "test_boris_uniform_b_rotation", {})]),
    ("Boris: s = t / (1 + t^2) (factor 2 dropped)",
     "sv[d] = 2.0 * t[d] / (1.0 + t2);", "sv[d] = t[d] / (1.0 + t2);",
     [("test_oracle_particles", "test_boris_uniform_b_rotation", {})]),
    ("Boris: t without the Lorentz factor",
     "t[d] = eps * b[d] / gm;", "t[d] = eps * b[d];",
     [("test_oracle_particles", "test_boris_uniform_b_rotation", {}),
      ("test_oracle_particles", "test_boris_orbit_radius_through_step", {})]),
    ("Esirkepov 3D: DSy DSz / 2 instead of / 3 in Wx",
     "0.5 * S0[1][b] * DS[2][c] + DS[1][b] * DS[2][c] / 3.0);",
     "0.5 * S0[1][b] * DS[2][c] + DS[1][b] * DS[2][c] / 2.0);",
     [("test_oracle_particles", "test_esirkepov_continuity_and_total_current", {"dim": 3, "order": 1})]),
    ("Esirkepov 2D: Jz weight S0x + DSx (half dropped)",
     "acc += DS[2][c] * (S0[0][a] + 0.5 * DS[0][a]);", "acc += DS[2][c] * (S0[0][a] + DS[0][a]);",
     [("test_oracle_particles", "test_esirkepov_continuity_and_total_current", {"dim": 2, "order": 1})]),
    ("Esirkepov: sign of the z current factor",
     "const double cz = -qw * s->hz / (s->dt * vol);", "const double cz = qw * s->hz / (s->dt * vol);",
     [("test_oracle_particles", "test_esirkepov_continuity_and_total_current", {"dim": 2, "order": 1})]),
    ("electron push: force of a positive charge",
     "opic_boris(u, eb, eb + 3, -1.0, s->dt);", "opic_boris(u, eb, eb + 3, 1.0, s->dt);",
     [("test_oracle_physics", "test_cold_plasma_oscillation", {})]),
    ("electron push: deposit with the ion's sign",
     "opic_deposit_current(s, -p->a[OPIC_PW][n], x0, x1, u[1] / g);",
     "opic_deposit_current(s, p->a[OPIC_PW][n], x0, x1, u[1] / g);",
     [("test_oracle_physics", "test_cold_plasma_oscillation", {}),
      ("test_oracle_physics", "test_continuity_through_the_loop", {"dim": 2, "order": 1, "npass": 1})]),
    ("filter: weights (1/4, 1/2, 1/2)",
     "0.25 * lo + 0.5 * tmp[fidx(s, i, j, k)] + 0.25 * hi;", "0.25 * lo + 0.5 * tmp[fidx(s, i, j, k)] + 0.5 * hi;",
     [("test_oracle_fields", "test_filter_transfer_function", {})]),
    ("filter: absorbing z end mirrored instead of zero",
     "lo = k > 0 ? tmp[fidx(s, i, j, k - 1)] : 0.0;", "lo = k > 0 ? tmp[fidx(s, i, j, k - 1)] : tmp[fidx(s, i, j, k)];",
     [("test_oracle_fields", "test_filter_absorbing_z_boundary_and_dc", {})]),
    ("filter: y passes skipped in 3D",
     "if (ax == 1 && s->g.dim != 3)", "if (ax == 1)",
     [("test_oracle_fields", "test_filter_transfer_function", {}),
      ("test_oracle_physics", "test_continuity_through_the_loop", {"dim": 3, "order": 1, "npass": 1})]),
    ("Yee: sign of dEy/dz in the Bx update",
     "Bx[o] -= h * (dEz_dy - dEy_dz);", "Bx[o] -= h * (dEz_dy + dEy_dz);",
     [("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 3, "pol": "A"}),
      ("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 3, "pol": "B"}),
      ("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 2, "pol": "TE"}),
      ("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 2, "pol": "TM"})]),
    ("Yee: current term pi J instead of 2 pi J in Ez",
     "Ez[o] += dt * ((dBy_dx - dBx_dy) - TWO_PI * Jz[o]);", "Ez[o] += dt * ((dBy_dx - dBx_dy) - PI_ * Jz[o]);",
     [("test_oracle_physics", "test_cold_plasma_oscillation", {}),
      ("test_oracle_physics", "test_continuity_through_the_loop", {"dim": 2, "order": 1, "npass": 1})]),
    ("Yee: dBz/dx taken forward instead of backward in Ey",
     "double dBz_dx = (Bz[o] - Bz[fidx(s, im, j, k)]) / s->hx;",
     "double dBz_dx = (Bz[fidx(s, (i + 1) % nx, j, k)] - Bz[o]) / s->hx;",
     [("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 2, "pol": "TE"}),
      ("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 2, "pol": "TM"})]),
    ("Yee: full instead of half B steps",
     "        yee_b(s, 0.5 * s->dt);\n        yee_e(s);\n        yee_b(s, 0.5 * s->dt);",
     "        yee_b(s, s->dt);\n        yee_e(s);\n        yee_b(s, 0.5 * s->dt);",
     [("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 2, "pol": "TE"}),
      ("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 2, "pol": "TM"})]),
    ("Mur: coefficient of the wrong sign",
     "const double cm = (dt - s->hz) / (dt + s->hz);", "const double cm = (s->hz - dt) / (dt + s->hz);",
     [("test_oracle_fields", "test_mur_absorbs_normal_pulse", {"pol": 0}),
      ("test_oracle_fields", "test_mur_absorbs_normal_pulse", {"pol": 1})]),
    ("antenna: sheet current 1/(2 pi hz)",
     "const double j0 = -amp / (PI_ * s->hz);", "const double j0 = -amp / (TWO_PI * s->hz);",
     [("test_oracle_fields", "test_antenna_amplitude_and_carrier", {})]),
    ("antenna: no Doppler factor in the boosted frame",
     "const double D = 1.0 / (s->gam * (1.0 + s->beta));", "const double D = 1.0;",
     [("test_oracle_physics", "test_boosted_antenna_doppler", {})]),
    ("antenna: waist taken as exp(-r^2 / (2 w0^2))",
     "exp(-r2 / (l->waist * l->waist))", "exp(-r2 / (2.0 * l->waist * l->waist))",
     [("test_oracle_fields", "test_antenna_beam_has_the_waist", {"pol": 0}),
      ("test_oracle_fields", "test_antenna_beam_has_the_waist", {"pol": 1})]),
    ("boosted load: weight without the density's factor gamma",
     "const double wfac = s->gam * vol / (double)(ppx * ppy * ppz);",
     "const double wfac = vol / (double)(ppx * ppy * ppz);",
     [("test_oracle_physics", "test_boosted_load_density_and_contraction", {})]),
    ("boosted load: lab z not contracted",
     "const double zb = zlab / s->gam - s->beta * s->t - opic_window(s);",
     "const double zb = zlab - s->beta * s->t - opic_window(s);",
     [("test_oracle_physics", "test_boosted_load_density_and_contraction", {})]),
    ("injection: plasma entering a step late",
     "static void inject(opic *s) { inject_at(s, s->t + s->dt); }",
     "static void inject(opic *s) { inject_at(s, s->t); }",
     [("test_oracle_physics", "test_boosted_injection_flux_and_positions", {}),
      ("test_oracle_physics", "test_injected_plasma_matches_free_drift", {})]),
    ("snapshots: event time gamma (T + beta Z)",
     "const double tp = gam * (T - beta * Z);", "const double tp = gam * (T + beta * Z);",
     [("test_oracle_btd", "test_snapshot_coverage", {}),
      ("test_oracle_btd", "test_lab_and_boosted_runs_of_one_pulse_agree", {})]),
    ("snapshots: Ex = gamma (Ex' - beta By')",
     "const double lab[6] = {gam * (e[0] + beta * e[4])", "const double lab[6] = {gam * (e[0] - beta * e[4])",
     [("test_oracle_btd", "test_static_fields_seen_from_the_lab", {"e": (0.0, 0.0, 0.0), "b": (0.4, 0.9, -0.2)}),
      ("test_oracle_btd", "test_lab_and_boosted_runs_of_one_pulse_agree", {})]),
    ("diagnostics: field energy without the 1/2",
     "out[0] = 0.5 * vol * fe.s;", "out[0] = vol * fe.s;",
     [("test_oracle_diagnostics", "test_field_energy_of_modes_and_uniform_fields", {"dim": 2, "bc_z": 1})]),
    ("diagnostics: u^2 / gamma instead of gamma - 1",
     "(u2 / (sqrt(1.0 + u2) + 1.0))", "(u2 / sqrt(1.0 + u2))",
     [("test_oracle_diagnostics", "test_kinetic_energy_and_charge_of_a_cold_plasma", {"gam": 13.0})]),
    ("diagnostics: plain instead of compensated sum",
     "k->c = (t - k->s) - y;", "k->c = 0.0;",
     [("test_oracle_diagnostics", "test_field_energy_sum_is_compensated", {})]),
    ("lab view: By = gamma (By' - beta Ex')",
     "case OPIC_BY: v = gam * (s->f[OPIC_BY][o] + beta", "case OPIC_BY: v = gam * (s->f[OPIC_BY][o] - beta",
     [("test_oracle_diagnostics", "test_lab_fields_of_uniform_fields", {"gam": 3.0})]),
    ("moving window: fields shifted by S - 1 planes",
     "f[k * plane + o] = k + S <= s->g.nz ? f[(k + S) * plane + o] : 0.0;",
     "f[k * plane + o] = k + S <= s->g.nz ? f[(k + S - 1) * plane + o] : 0.0;",
     [("test_oracle_window", "test_pulse_in_window_matches_long_box", {})]),
    ("ion push: deposit with the electron's sign",
     "opic_deposit_current(s, p->a[OPIC_PW][n], x0, x1, u[1] / g);",
     "opic_deposit_current(s, -p->a[OPIC_PW][n], x0, x1, u[1] / g);",
     [("test_oracle_physics", "test_boosted_plasma_without_laser_stays_field_free", {})]),
    ("ion push: half the drift per step",
     "x1[2] = x0[2] + s->dt * u[2] / g;\n        opic_deposit_current(s, p->a",
     "x1[2] = x0[2] + 0.5 * s->dt * u[2] / g;\n        opic_deposit_current(s, p->a",
     [("test_oracle_physics", "test_boosted_plasma_without_laser_stays_field_free", {})]),
    ("injection: the ions of the entering plasma left out",
     "            if (s->has_ions)\n                species_push(&s->sp[1], q->x, q->y, zb, 0.0, 0.0, uz0, q->w, q->id);\n",
     "",
     [("test_oracle_physics", "test_boosted_injection_flux_and_positions", {}),
      ("test_oracle_physics", "test_boosted_plasma_without_laser_stays_field_free", {})]),
    ("lattice jitter: U(0, J) instead of U(-J, J) in x",
     "(p->jitter * s->hx) * (2.0 * opic_uniform(s->g.seed, c0) - 1.0)",
     "(p->jitter * s->hx) * opic_uniform(s->g.seed, c0)",
     [("test_oracle_physics", "test_lattice_jitter_is_symmetric_and_bounded", {})]),
    ("density ramp: half its slope",
     "r = (z - p->z_start) / p->ramp;", "r = 0.5 * (z - p->z_start) / p->ramp;",
     [("test_oracle_basics", "test_density_profile", {})]),
    ("boosted frame: cells stretched by gamma instead of gamma (1 + beta)",
     "s->hz = g->dz * (s->gam * (1.0 + s->beta));", "s->hz = g->dz * s->gam;",
     [("test_oracle_physics", "test_boosted_load_density_and_contraction", {}),
      ("test_oracle_physics", "test_boosted_antenna_doppler", {})]),
    ("time step in 3D without the y cell",
     "s->dt = g->cfl / sqrt(1.0 / (s->hx * s->hx) + 1.0 / (s->hy * s->hy) + 1.0 / (s->hz * s->hz));",
     "s->dt = g->cfl / sqrt(1.0 / (s->hx * s->hx) + 1.0 / (s->hz * s->hz));",
     [("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 3, "pol": "A"}),
      ("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 3, "pol": "B"})]),
    ("Boris: second half of the electric impulse dropped",
     "u[d] = upl[d] + eps * e[d];", "u[d] = upl[d];",
     [("test_oracle_particles", "test_boris_uniform_e", {})]),
    ("Esirkepov: window starting at the lower cell instead of one below",
     "lo[d] = (int64_t)floor(a < b ? a : b) - 1;", "lo[d] = (int64_t)floor(a < b ? a : b);",
     [("test_oracle_particles", "test_esirkepov_continuity_and_total_current", {"dim": 2, "order": 2})]),
    ("Esirkepov 2D: out-of-plane current without 1/V",
     "const double cyv = qw * vy / vol;", "const double cyv = qw * vy;",
     [("test_oracle_particles", "test_esirkepov_continuity_and_total_current", {"dim": 2, "order": 1})]),
    ("charge density without 1/V",
     "const double qw = q * p->a[OPIC_PW][n] / vol;", "const double qw = q * p->a[OPIC_PW][n];",
     [("test_oracle_physics", "test_continuity_through_the_loop", {"dim": 2, "order": 1, "npass": 1})]),
    ("valid z planes: half-integer components given the top plane too",
     "return sz > 0.0 ? s->g.nz - 1 : s->g.nz;", "return s->g.nz;",
     [("test_oracle_fields", "test_filter_absorbing_z_boundary_and_dc", {}),
      ("test_oracle_diagnostics", "test_field_energy_of_modes_and_uniform_fields", {"dim": 2, "bc_z": 1})]),
    ("antenna: Jx sheet at integer x",
     "const double sx = l->pol == 0 ? 0.5 : 0.0;", "const double sx = 0.0;",
     [("test_oracle_fields", "test_antenna_beam_has_the_waist", {"pol": 0})]),
    ("lab view: partner taken from one plane instead of the mean of two",
     "return 0.5 * (f[fidx(s, i, j, a)] + f[fidx(s, i, j, b)]);", "return f[fidx(s, i, j, b)];",
     [("test_oracle_diagnostics", "test_lab_fields_pair_each_component_with_its_staggered_partner", {})]),
    ("snapshots: z interpolation weights swapped",
     "*out = (1.0 - fz) * f[fidx(s, i, j, k)] + fz * f[fidx(s, i, j, k + 1)];",
     "*out = fz * f[fidx(s, i, j, k)] + (1.0 - fz) * f[fidx(s, i, j, k + 1)];",
     [("test_oracle_btd", "test_lab_and_boosted_runs_of_one_pulse_agree", {})]),
    ("moving window: particles shifted one cell short",
     "p->a[OPIC_PZ][k] -= dz;", "p->a[OPIC_PZ][k] -= dz - s->hz;",
     [("test_oracle_window", "test_static_plasma_through_window_is_the_lattice", {})]),
    ("uniform deviate from 52 instead of 53 bits (values in [0, 1/2))",
     "return (double)(opic_splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0);",
     "return (double)(opic_splitmix64(seed, counter) >> 12) * (1.0 / 9007199254740992.0);",
     [("test_oracle_physics", "test_lattice_jitter_is_symmetric_and_bounded", {})]),
    ("Mur at the top end: old planes swapped",
     "Ex[(int64_t)nz * plane + q] = exm + cm * (Ex[(int64_t)(nz - 1) * plane + q] - exn);",
     "Ex[(int64_t)nz * plane + q] = exn + cm * (Ex[(int64_t)(nz - 1) * plane + q] - exm);",
     [("test_oracle_fields", "test_mur_absorbs_normal_pulse", {"pol": 0}),
      ("test_oracle_fields", "test_mur_absorbs_normal_pulse", {"pol": 1})]),
    ("antenna: sheet evaluated at t^n instead of t^{n+1/2}",
     "const double th = s->t + 0.5 * s->dt;", "const double th = s->t;",
     [("test_oracle_fields", "test_antenna_carrier_phase_and_plane", {})]),
    ("antenna: plane below z_antenna instead of the nearest",
     "int ka = (int)floor(l->z_antenna / s->hz + 0.5);", "int ka = (int)floor(l->z_antenna / s->hz);",
     [("test_oracle_fields", "test_antenna_carrier_phase_and_plane", {})]),
    ("antenna: FWHM read as the field's instead of the intensity's",
     "const double tau = l->fwhm / sqrt(2.0 * log(2.0));", "const double tau = l->fwhm / (2.0 * sqrt(log(2.0)));",
     [("test_oracle_fields", "test_antenna_amplitude_and_carrier", {})]),
    ("Yee 3D: sign of dBx/dy in the Ez update",
     "double dBx_dy = dim3 ? (Bx[o] - Bx[fidx(s, i, jm, k)]) / s->hy : 0.0;\n                    Ez",
     "double dBx_dy = dim3 ? (Bx[fidx(s, i, jm, k)] - Bx[o]) / s->hy : 0.0;\n                    Ez",
     [("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 3, "pol": "A"}),
      ("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 3, "pol": "B"})]),
    ("Esirkepov 3D: DSx S0y / 2 dropped from Wz",
     "acc += DS[2][c] * (S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b] +",
     "acc += DS[2][c] * (S0[0][a] * S0[1][b] +",
     [("test_oracle_particles", "test_esirkepov_continuity_and_total_current", {"dim": 3, "order": 1})]),
    ("snapshots: Bx = gamma (Bx' + beta Ey')",
     "gam * (e[3] - beta * e[1])", "gam * (e[3] + beta * e[1])",
     [("test_oracle_btd", "test_static_fields_seen_from_the_lab", {"e": (0.3, -0.7, 0.25), "b": (0.0, 0.0, 0.0)})]),
    ("moving window: plasma it moves over placed a step ahead",
     "    inject_at(s, s->t);\n    /* the plasma the window", "    inject_at(s, s->t + s->dt);\n    /* the plasma the window",
     [("test_oracle_window", "test_boosted_plasma_through_window_matches_long_box", {})]),
    ("electron push: particles past the top end kept",
     "        } else if (x1[2] < 0.0 || x1[2] >= s->Lz) {\n            species_remove(p, n);\n            continue;\n"
     "        }\n        p->a[OPIC_PX][n] = x1[0];\n        p->a[OPIC_PY][n] = x1[1];\n        p->a[OPIC_PZ][n] = x1[2];\n"
     "        ++n;\n    }\n}\n\n/* ions",
     "        } else if (x1[2] < 0.0) {\n            species_remove(p, n);\n            continue;\n"
     "        }\n        p->a[OPIC_PX][n] = x1[0];\n        p->a[OPIC_PY][n] = x1[1];\n        p->a[OPIC_PZ][n] = x1[2];\n"
     "        ++n;\n    }\n}\n\n/* ions",
     [("test_oracle_particles", "test_particles_leaving_through_absorbing_ends_are_removed", {"sp": 0})]),
    ("ion move: particles past the bottom end kept",
     "        } else if (x1[2] < 0.0 || x1[2] >= s->Lz) {\n            species_remove(p, n);\n            continue;\n"
     "        }\n        p->a[OPIC_PX][n] = x1[0];\n        p->a[OPIC_PY][n] = x1[1];\n        p->a[OPIC_PZ][n] = x1[2];\n"
     "        ++n;\n    }\n}\n\n/* ------",
     "        } else if (x1[2] >= s->Lz) {\n            species_remove(p, n);\n            continue;\n"
     "        }\n        p->a[OPIC_PX][n] = x1[0];\n        p->a[OPIC_PY][n] = x1[1];\n        p->a[OPIC_PZ][n] = x1[2];\n"
     "        ++n;\n    }\n}\n\n/* ------",
     [("test_oracle_particles", "test_particles_leaving_through_absorbing_ends_are_removed", {"sp": 1}),
      ("test_oracle_physics", "test_boosted_plasma_without_laser_stays_field_free", {})]),
    ("boosted load: ion weight halved",
     "species_push(&s->sp[1], x, y, zb, 0.0, 0.0, uz0, w, L);", "species_push(&s->sp[1], x, y, zb, 0.0, 0.0, uz0, 0.5 * w, L);",
     [("test_oracle_physics", "test_boosted_plasma_without_laser_stays_field_free", {}),
      ("test_oracle_diagnostics", "test_kinetic_energy_and_charge_of_a_cold_plasma", {"gam": 13.0})]),
    ("lattice points at the cell's corner instead of its centre",
     "double x = ((double)ix + 0.5) * (s->hx / (double)ppx) +", "double x = ((double)ix) * (s->hx / (double)ppx) +",
     [("test_oracle_physics", "test_lattice_jitter_is_symmetric_and_bounded", {})]),
    ("diagnostics: drifting ions counted with the electrons' charge",
     "kahan_add(&q, ion->a[OPIC_PW][p]);", "kahan_add(&q, -ion->a[OPIC_PW][p]);",
     [("test_oracle_diagnostics", "test_kinetic_energy_and_charge_of_a_cold_plasma", {"gam": 13.0})]),
    ("snapshots: no interpolation in time within the step",
     "const double th = (tp - t0) / s->dt;", "const double th = 0.0;",
     [("test_oracle_btd", "test_lab_and_boosted_runs_of_one_pulse_agree", {})]),
    ("lab plasma: immobile ions' background with the electrons' sign",
     "deposit_rho_species(s, &s->sp[0], 0, 1.0, s->rho_bg);", "deposit_rho_species(s, &s->sp[0], 0, -1.0, s->rho_bg);",
     [("test_oracle_physics", "test_plasma_with_its_ions_is_neutral", {"gam": 1.0})]),
    ("charge density: drifting ions with the electrons' sign",
     "        deposit_rho_species(s, &s->sp[1], 0, 1.0, rho);", "        deposit_rho_species(s, &s->sp[1], 0, -1.0, rho);",
     [("test_oracle_physics", "test_plasma_with_its_ions_is_neutral", {"gam": 5.0})]),
    ("moving window: first move as soon as it starts (one step of S ahead)",
     "s->win_v * (s->t - s->win_t0) >= (double)(s->win_n + 1) * s->win_S * s->hz",
     "s->win_v * (s->t - s->win_t0) >= (double)(s->win_n) * s->win_S * s->hz",
     [("test_oracle_window", "test_antenna_stays_put_as_the_window_moves", {})]),
    ("moving window: antenna carried along with the window",
     "const int64_t ka = s->ka - s->win_n * s->win_S;", "const int64_t ka = s->ka;",
     [("test_oracle_window", "test_antenna_stays_put_as_the_window_moves", {})]),
    ("Boris: rotation with gamma of u^{n-1/2} instead of u-",
     "const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);",
     "const double gm = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);",
     [("test_oracle_particles", "test_boris_step_satisfies_its_implicit_form", {})]),
    ("gather: periodic z wrapped over nz + 1 planes",
     "        if (s->g.bc_z == 0)\n            k = wrap_index(k, s->g.nz);\n        else if (k < 0 || k > zmax)\n"
     "            continue;\n        for (int cy",
     "        if (s->g.bc_z == 0)\n            k = wrap_index(k, s->g.nz + 1);\n        else if (k < 0 || k > zmax)\n"
     "            continue;\n        for (int cy",
     [("test_oracle_basics", "test_gather_wraps_periodic_boundaries", {"dim": 2, "order": 1})]),
    ("snapshots: event height not taken relative to the moving window",
     "const double zp = gam * (Z - beta * T) - opic_window(s);", "const double zp = gam * (Z - beta * T);",
     [("test_oracle_btd", "test_snapshots_of_a_windowed_run_match_the_long_box", {})]),
    ("antenna 3D: Jy sheet at integer y",
     "const double sy = (l->pol == 1 && s->g.dim == 3) ? 0.5 : 0.0;", "const double sy = 0.0;",
     [("test_oracle_fields", "test_antenna_beam_has_the_waist_across_y", {})]),
    ("snapshots: on-axis line taken at x = 0 instead of the middle column",
     "const int64_t i = nxs == 1 ? s->g.nx / 2 : is;", "const int64_t i = nxs == 1 ? 0 : is;",
     [("test_oracle_btd", "test_on_axis_snapshot_is_the_middle_column", {})]),
    ("filter: x neighbour two nodes away",
     "lo = tmp[fidx(s, wrap_index(i - 1, nx), j, k)];", "lo = tmp[fidx(s, wrap_index(i - 2, nx), j, k)];",
     [("test_oracle_fields", "test_filter_transfer_function", {}),
      ("test_oracle_fields", "test_filter_is_its_own_transpose", {"dim": 2, "bc": 1, "npass": 1})]),
    ("time step in 2D with half the z term",
     "s->dt = g->cfl / sqrt(1.0 / (s->hx * s->hx) + 1.0 / (s->hz * s->hz));",
     "s->dt = g->cfl / sqrt(1.0 / (s->hx * s->hx) + 0.5 / (s->hz * s->hz));",
     [("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 2, "pol": "TE"}),
      ("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 2, "pol": "TM"}),
      ("test_oracle_physics", "test_cold_plasma_oscillation", {})]),
    ("Yee: sign of dEx/dy in the Bz update",
     "Bz[o] -= h * (dEy_dx - dEx_dy);", "Bz[o] -= h * (dEy_dx + dEx_dy);",
     [("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 3, "pol": "A"}),
      ("test_oracle_fields", "test_yee_discrete_eigenmode", {"dim": 3, "pol": "B"})]),
    ("Mur at the bottom end: old planes swapped for Ey",
     "Ey[q] = ey1 + cm * (Ey[plane + q] - ey0);", "Ey[q] = ey0 + cm * (Ey[plane + q] - ey1);",
     [("test_oracle_fields", "test_mur_absorbs_normal_pulse", {"pol": 1})]),
    ("injection: entering ions at rest instead of drifting",
     "                species_push(&s->sp[1], q->x, q->y, zb, 0.0, 0.0, uz0, q->w, q->id);",
     "                species_push(&s->sp[1], q->x, q->y, zb, 0.0, 0.0, 0.0, q->w, q->id);",
     [("test_oracle_physics", "test_injected_plasma_matches_free_drift", {}),
      ("test_oracle_physics", "test_boosted_plasma_without_laser_stays_field_free", {})]),
    ("lab view: By's partner Ex taken from the planes below",
     "case OPIC_BY: v = gam * (s->f[OPIC_BY][o] + beta * zmean(s, s->f[OPIC_EX], OPIC_EX, i, j, k, 1)); break;",
     "case OPIC_BY: v = gam * (s->f[OPIC_BY][o] + beta * zmean(s, s->f[OPIC_EX], OPIC_EX, i, j, k, 0)); break;",
     [("test_oracle_diagnostics", "test_lab_fields_pair_each_component_with_its_staggered_partner", {})]),
    ("moving window: particles within a cell of the bottom removed too",
     "            if (p->a[OPIC_PZ][k] < 0.0)\n                species_remove(p, k);",
     "            if (p->a[OPIC_PZ][k] < s->hz)\n                species_remove(p, k);",
     [("test_oracle_window", "test_static_plasma_through_window_is_the_lattice", {}),
      ("test_oracle_window", "test_boosted_plasma_through_window_matches_long_box", {})]),
    ("gather 3D: y support starting at the particle's cell (quadratic node below lost)",
     "        by = (int64_t)floor(yi) - 1;\n        ny_loop = 4;", "        by = (int64_t)floor(yi);\n        ny_loop = 4;",
     [("test_oracle_basics", "test_gather_reproduces_linear_fields", {"dim": 3, "order": 2})]),
    ("moving window: the ions' background left where it was",
     "    bufs[OPIC_NCOMP] = s->rho_bg;\n    for (int c = 0; c <= OPIC_NCOMP; ++c) {",
     "    bufs[OPIC_NCOMP] = s->rho_bg;\n    for (int c = 0; c < OPIC_NCOMP; ++c) {",
     [("test_oracle_window", "test_lab_plasma_with_immobile_ions_stays_neutral_through_the_window", {})]),
    ("moving window: the covered plasma brought in without its ions' background",
     "    if (s->bg_ions)\n        deposit_rho_species(s, &s->sp[0], n0, 1.0, s->rho_bg);", "",
     [("test_oracle_window", "test_lab_plasma_with_immobile_ions_stays_neutral_through_the_window", {})]),
    ("antenna: envelope peak at 2 tau instead of 3 tau",
     "const double spk = l->t_peak >= 0.0 ? l->t_peak : 3.0 * tau;",
     "const double spk = l->t_peak >= 0.0 ? l->t_peak : 2.0 * tau;",
     [("test_oracle_fields", "test_antenna_amplitude_and_carrier", {})]),
    ("antenna: polarisations swapped",
     "const int c = l->pol == 0 ? OPIC_JX : OPIC_JY;", "const int c = l->pol == 0 ? OPIC_JY : OPIC_JX;",
     [("test_oracle_fields", "test_antenna_amplitude_and_carrier", {})]),
    ("antenna: allowed on plane 1",
     "    if (ka < 2)\n        ka = 2;\n    if (ka > s->g.nz - 2)", "    if (ka < 1)\n        ka = 1;\n    if (ka > s->g.nz - 2)",
     [("test_oracle_fields", "test_antenna_amplitude_and_carrier", {})]),
    ("antenna: default centre half a cell off the box's middle",
     "        s->las.xc = 0.5 * s->Lx;", "        s->las.xc = 0.5 * s->Lx + 0.5 * s->hx;",
     [("test_oracle_fields", "test_antenna_beam_has_the_waist", {"pol": 0})]),
    ("Mur: old E taken from plane nz - 2",
     "const int planes[4] = {0, 1, nz - 1, nz};", "const int planes[4] = {0, 1, nz - 2, nz};",
     [("test_oracle_fields", "test_mur_absorbs_normal_pulse", {"pol": 1})]),
    ("filter: every component given the integer-z planes",
     "    const int zmax = zmax_of(s, STAG[c][2]);\n    memcpy(tmp", "    const int zmax = zmax_of(s, 0.0);\n    memcpy(tmp",
     [("test_oracle_fields", "test_filter_absorbing_z_boundary_and_dc", {})]),
    ("Boris: second half impulse subtracted",
     "        u[d] = upl[d] + eps * e[d];", "        u[d] = upl[d] - eps * e[d];",
     [("test_oracle_particles", "test_boris_uniform_e", {})]),
    ("diagnostics: electrons counted with positive charge",
     "        kahan_add(&q, -e->a[OPIC_PW][p]);", "        kahan_add(&q, e->a[OPIC_PW][p]);",
     [("test_oracle_diagnostics", "test_kinetic_energy_and_charge_of_a_cold_plasma", {"gam": 13.0})]),
    ("snapshots: points marked filled although a component was out of range",
     "            if (ok)\n                s->btd_fill[(size_t)js * b->nz + k] = 1;",
     "            s->btd_fill[(size_t)js * b->nz + k] = 1;",
     [("test_oracle_btd", "test_snapshot_coverage", {})]),
]


def _module(name: str, path: str):
    # a fresh instance of a module file (registered, as dataclasses need)
    spec = importlib.util.spec_from_file_location(name, path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def source():
    with open(os.path.join(ORACLE, "pic_oracle.c")) as f:
        return f.read()


def test_every_planted_text_occurs_once(source):
    for what, old, new, pins in CASES:
        assert source.count(old) == 1, what
        assert old != new and pins, what


def _run_pins(source: str, tmp_path, tag: str, pins) -> list:
    """Compile `source` as the oracle, run the pins against it and return
    the names of those that failed."""
    src = tmp_path / "pic_oracle.c"
    src.write_text(source)
    so = str(tmp_path / "liboracle_planted.so")
    # the oracle's own flags (oracle.build_oracle)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-I", ORACLE, "-o", so, str(src), "-lm"], check=True)
    O = _module(f"oracle_planted_{tag}", os.path.join(ORACLE, "oracle.py"))
    O.build_oracle = lambda force=False: so
    failed = []
    for fname, test, params in pins:
        fn = getattr(_module(f"pins_{fname}_{tag}", os.path.join(TESTS, fname + ".py")), test)
        try:
            fn(O, **params)
        except (AssertionError, ArithmeticError, ValueError, RuntimeError):
            # a failed check, or arithmetic (a fit, a bound) the pin cannot
            # even complete on the planted copy
            failed.append(test)
    # the pins ran on the compiled copy, not on the oracle's own build
    assert O._lib is not None and O._lib._name == so
    return failed


def test_unplanted_copy_passes_every_pin(source, tmp_path):
    # the same harness on an unchanged copy: every pin used below passes
    pins, seen = [], set()
    for _, _, _, ps in CASES:
        for fname, test, params in ps:
            key = (fname, test, tuple(sorted(params.items())))
            if key not in seen:
                seen.add(key)
                pins.append((fname, test, params))
    assert _run_pins(source + "\n/* unchanged */\n", tmp_path, "control", pins) == []


@pytest.mark.filterwarnings("ignore::RuntimeWarning")   # (overflow in a pin's fit on an unstable copy)
@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(source, tmp_path, case):
    what, old, new, pins = CASES[case]
    assert _run_pins(source.replace(old, new, 1), tmp_path, str(case), pins), f"no pin caught: {what}"
