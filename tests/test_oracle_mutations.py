"""Planted mistakes in the oracle, each caught by the oracle's own pins.

Each case copies ``oracle/grmhd_oracle.c``, replaces one expression with a plausible
wrong one (a dropped term, a wrong sign, factor, index or weight), compiles the copy
with the oracle's flags and runs the oracle's pin tests against it in a child process
(``GRMHD_ORACLE_LIB`` points the oracle at the copy).  Every case must make a pin
fail: a mistake of that kind anywhere in these parts of the oracle would not go
unnoticed.  The pins are the closed forms, paper tables, exact solutions, invariants
and symmetries of test_oracle_cell.py, test_oracle_physics.py,
test_oracle_diagnostics.py, test_oracle_ppm.py and test_oracle_ideal_emf.py (its two
slowest convergence runs left out, except for mistakes in the ideal-limit EMF, which
run that file whole); mistakes in the GLM variant run test_oracle_glm.py."""
import concurrent.futures as cf
import os
import subprocess
import sys

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "grmhd_oracle.c")
PINS = ["tests/test_oracle_cell.py", "tests/test_oracle_diagnostics.py", "tests/test_oracle_physics.py",
        "tests/test_oracle_ppm.py", "tests/test_oracle_ideal_emf.py"]
SKIP = ["tests/test_oracle_ideal_emf.py::test_ideal_and_resistive_emf_agree_in_the_stiff_limit",
        "tests/test_oracle_ideal_emf.py::test_ideal_emf_advects_the_loop_at_second_order"]

# the pins of the GLM variant and of the ideal-limit EMF (all of them)
GLM_PINS = ["tests/test_oracle_glm.py"]
IDEAL_PINS = ["tests/test_oracle_ideal_emf.py"]

# (name, expression in the oracle, the mistake put in its place[, pins if not PINS])
MUTATIONS = [
    # prim2con (Sec. 2.1): tau without -D; the sign of the Poynting term in S
    ("tau_without_D",
     "double tau = rho * h * W * W - p + 0.5 * (E2 + B2) - D;",
     "double tau = rho * h * W * W - p + 0.5 * (E2 + B2);"),
    ("S_poynting_sign",
     "S[j] = rho * h * W * W * v_lo[j] + sg * exb;",
     "S[j] = rho * h * W * W * v_lo[j] - sg * exb;"),
    # implicit E(u) and residual (Sec. 2.4)
    ("A5_sign",
     "double A5 = -1.0 - x2 * W / p;",
     "double A5 = 1.0 - x2 * W / p;"),
    # the dynamo terms of the A_k (Sec. 2.4 with xi != 0)
    ("A0_dynamo_term",
     "double A0 = W + et + x2 * (W * W - 1.0) / p;",
     "double A0 = W + et + x2 * (W * W + 1.0) / p;"),
    ("A1_dynamo_term",
     "double A1 = et / q + x2 * et * W / (p * q);",
     "double A1 = et / q - x2 * et * W / (p * q);"),
    ("A2_sign",
     "double A2 = -xi * et / p;",
     "double A2 = xi * et / p;"),
    ("A3_swapped",
     "double A3 = xi * q / p;",
     "double A3 = xi * p / q;"),
    ("A4_eta_sign",
     "double A4 = xi * (1.0 - et * et + x2) / (p * q);",
     "double A4 = xi * (1.0 + et * et + x2) / (p * q);"),
    ("residual_ExB_sign",
     "f[i] = wt * u_lo[i] - (c->S[i] - eEB[i]);",
     "f[i] = wt * u_lo[i] - (c->S[i] + eEB[i]);"),
    ("wtilde_U_sign",
     "double wt = (W * (c->tau + c->D - U) - c->D / Gh) / den;",
     "double wt = (W * (c->tau + c->D + U) - c->D / Gh) / den;"),
    ("jacobian_dU_sign",
     "dwt[j] = ((c->tau + c->D - U) * u_lo[j] / W - 2.0 * wt * u_lo[j] - W * dU) / den;",
     "dwt[j] = ((c->tau + c->D - U) * u_lo[j] / W - 2.0 * wt * u_lo[j] + W * dU) / den;"),
    # reconstruction (Sec. 5 MC; PPM)
    ("mc_centred_factor",
     "return minmod3(2.0 * (u0 - um), 0.5 * (up - um), 2.0 * (up - u0));",
     "return minmod3(2.0 * (u0 - um), (up - um), 2.0 * (up - u0));"),
    ("minmod_picks_max",
     "if (a > 0 && b > 0 && c > 0) return fmin(a, fmin(b, c));",
     "if (a > 0 && b > 0 && c > 0) return fmax(a, fmax(b, c));"),
    ("ppm_slope_weight",
     "return a0 + 0.5 * (ap - a0) - (mc_slope(a0, ap, app) - mc_slope(am, a0, ap)) / 6.0;",
     "return a0 + 0.5 * (ap - a0) - (mc_slope(a0, ap, app) - mc_slope(am, a0, ap)) / 3.0;"),
    # physical fluxes and HLL (Sec. 2.1, Sec. 2.5)
    ("D_flux_wrong_index",
     "F[0] = sg * D * alp * v[d];",
     "F[0] = sg * D * alp * v[(d + 1) % 3];"),
    ("maxwell_stress_sign",
     "- pr[5 + d] * E_lo[j] - B[d] * B_lo[j]);",
     "- pr[5 + d] * E_lo[j] + B[d] * B_lo[j]);"),
    ("E_flux_sign",
     "for (int k = 0; k < 3; k++) s += levi(d, j, k) * alp * B_lo[k];",
     "for (int k = 0; k < 3; k++) s -= levi(d, j, k) * alp * B_lo[k];"),
    ("hll_diffusion_sign",
     "for (int v = 0; v < NQ; v++)\n                F[d][v][c] = (cp * FL[v] + cm * FR[v] - cp * cm * (qR[v] - qL[v]))",
     "for (int v = 0; v < NQ; v++)\n                F[d][v][c] = (cp * FL[v] + cm * FR[v] + cp * cm * (qR[v] - qL[v]))"),
    # flux divergence and sources (Sec. 2.1)
    ("divergence_sign",
     "for (int v = 0; v < NQ; v++) Lc[v] -= (F[d][v][cp1] - F[d][v][c]) / g->dx[d];",
     "for (int v = 0; v < NQ; v++) Lc[v] += (F[d][v][cp1] - F[d][v][c]) / g->dx[d];"),
    ("gauss_law_half",
     "divqE += (qEp - qEm) / (2.0 * g->dx[d]);",
     "divqE += (qEp - qEm) / (g->dx[d]);"),
    ("lapse_source_sign",
     "Lc[1 + i] += al * sg * (-T00 * al * dal + 0.5 * tr);",
     "Lc[1 + i] += al * sg * (T00 * al * dal + 0.5 * tr);"),
    # upwind constrained transport (Sec. 3.2)
    ("uct_diffusion_sign",
     "+ cap * cam / (cap + cam) * (qBbR - qBbL)",
     "- cap * cam / (cap + cam) * (qBbR - qBbL)"),
    ("ct_update_sign",
     "if (g->act[fb]) r -= (Eh[fc][shift(g, c, fb, 1)] - Eh[fc][c]) / g->dx[fb];",
     "if (g->act[fb]) r += (Eh[fc][shift(g, c, fb, 1)] - Eh[fc][c]) / g->dx[fb];"),
    # IMEX stage assembly (Sec. 2.3): the implicit increment left out of the next base
    ("stage_base_without_R",
     "if (v >= 5) qs[v][c] += dt * a_ * Rs[j][v - 5][c];",
     "(void)a_;"),
    # diagnostics (Sec. 3.2 div B, the totals)
    ("divb_without_dx",
     "if (G.act[d]) dv += (bf[d][shift(&G, c, d, 1)] - bf[d][c]) / G.dx[d];",
     "if (G.act[d]) dv += (bf[d][shift(&G, c, d, 1)] - bf[d][c]);"),
    ("totals_without_volume",
     "for (int v = 0; v < NQ; v++) out[v] += q[v][c] * dV;",
     "for (int v = 0; v < NQ; v++) out[v] += q[v][c];"),
    # time step (Sec. 2.5): the speed alpha sqrt(gamma^dd) with the wrong power of psi
    ("dt_psi_power",
     "if (G.act[d]) s += alp_at(alp, c) * sqrt(1.0 / pow(ps, 4)) / G.dx[d];",
     "if (G.act[d]) s += alp_at(alp, c) * sqrt(1.0 / pow(ps, 2)) / G.dx[d];"),
    # implicit stage (Sec. 2.4, reading c2): eta_t without the lapse; R without 1/(a_ii dt)
    ("etat_without_lapse",
     "cl.etat = a_dt > 0 ? et / (alp_at(alp, c) * a_dt) : -1.0;",
     "cl.etat = a_dt > 0 ? et / a_dt : -1.0;"),
    ("R_without_a_dt",
     "if (R) R[i][c] = a_dt > 0 ? (qEn - q[5 + i][c]) / a_dt : 0.0;",
     "if (R) R[i][c] = a_dt > 0 ? (qEn - q[5 + i][c]) : 0.0;"),
    # cell-centred B (reading c11), the initial curl (Sec. 4), the tau source, the final
    # combination of the face fields
    ("cell_B_lower_face_only",
     "qBc[d][c] = 0.5 * (bf[d][c] + bf[d][shift(g, c, d, 1)]);",
     "qBc[d][c] = bf[d][c];"),
    ("curl_sign",
     "if (G.act[fb]) r += (A[fc][shift(&G, c, fb, 1)] - A[fc][c]) / G.dx[fb];",
     "if (G.act[fb]) r -= (A[fc][shift(&G, c, fb, 1)] - A[fc][c]) / G.dx[fb];"),
    ("tau_source_sign",
     "Lc[4] += al * sg * (-(S_lo[i] / gg) / al * dal);",
     "Lc[4] += al * sg * ((S_lo[i] / gg) / al * dal);"),
    ("face_combination_weight",
     "for (int d = 0; d < 3; d++) bf[d][c] += dt * wt[i] * Ls[i][NQ + d][c];",
     "for (int d = 0; d < 3; d++) bf[d][c] += dt * Ls[i][NQ + d][c];"),
    # metric factors (Sec. 2.1, Sec. 2.5, Sec. 3.2): the edge lapse as a sum, not a mean;
    # the tau flux without gamma^dd on S_d; d gamma_jj with the wrong power; rho_e not
    # undensitised; the E densitisation; the charge-current source's sign
    ("edge_lapse_sum",
     "ale /= nce;",
     "(void)nce;"),
    ("tau_flux_without_inverse_metric",
     "F[4] = sg * alp * (ginv * S_lo[d] - v[d] * D);",
     "F[4] = sg * alp * (S_lo[d] - v[d] * D);"),
    ("dgamma_factor",
     "double dgam = 4.0 * ps * ps * ps * dps;",
     "double dgam = 2.0 * ps * ps * ps * dps;"),
    ("rho_e_densitised",
     "double rhoe = divqE / sg;",
     "double rhoe = divqE;"),
    ("E_undensitised",
     "for (int j = 0; j < 3; j++) q[5 + j] = sg * pr[5 + j];",
     "for (int j = 0; j < 3; j++) q[5 + j] = pr[5 + j];"),
    ("charge_current_sign",
     "Lc[5 + i] += -sg * al * rhoe * v_up[i];",
     "Lc[5 + i] += sg * al * rhoe * v_up[i];"),
    # reconstruction: the left state's slope sign; PPM's second monotonicity branch
    ("mc_left_state_sign",
     "*L = a[m1] + 0.5 * mc_slope(a[m2], a[m1], a[c]);",
     "*L = a[m1] - 0.5 * mc_slope(a[m2], a[m1], a[c]);"),
    ("ppm_second_limit",
     "else if (-dd * dd > dd * m6) *aR = 3.0 * a0 - 2.0 * *aL;",
     "else if (-dd * dd > dd * m6) *aR = 3.0 * a0 - 2.0 * *aR;"),
    # GLM cleaning (Sec. 3.1): fluxes of q_B and q_Phi, their sources, densitisation
    ("glm_phi_flux_axis",
     "F[NQ + 3] = alp * sg * B[d];",
     "F[NQ + 3] = alp * sg * B[(d + 1) % 3];", GLM_PINS),
    ("glm_B_flux_sign",
     "for (int k = 0; k < 3; k++) s += levi(j, d, k) * alp * g * pr[5 + k];",
     "for (int k = 0; k < 3; k++) s -= levi(j, d, k) * alp * g * pr[5 + k];", GLM_PINS),
    ("glm_phi_densitisation",
     "q[NQ + 3] = sg * Phi;",
     "q[NQ + 3] = Phi;", GLM_PINS),
    ("glm_hll_diffusion_sign",
     "for (int v = 0; v < NGLM; v++)\n                F[d][v][c] = (cp * FL[v] + cm * FR[v] - cp * cm * (qR[v] - qL[v]))",
     "for (int v = 0; v < NGLM; v++)\n                F[d][v][c] = (cp * FL[v] + cm * FR[v] + cp * cm * (qR[v] - qL[v]))", GLM_PINS),
    ("glm_damping_sign",
     "Lc[NQ + 3] += -al * kappa * qPhi[c];",
     "Lc[NQ + 3] += al * kappa * qPhi[c];", GLM_PINS),
    ("glm_sB_without_inverse_metric",
     "Lc[NQ + i] += -sg * al * (1.0 / gg) * dPhi;",
     "Lc[NQ + i] += -sg * al * dPhi;", GLM_PINS),
    ("glm_dphi_factor",
     "double dPhi = (rec[NPR + 3][cp1] - rec[NPR + 3][cm1]) / (2.0 * g->dx[i]);",
     "double dPhi = (rec[NPR + 3][cp1] - rec[NPR + 3][cm1]) / (g->dx[i]);", GLM_PINS),
    ("glm_sphi_lapse_sign",
     "Lc[NQ + 3] += qB[i][c] * dal;",
     "Lc[NQ + 3] -= qB[i][c] * dal;", GLM_PINS),
    # ideal-limit edge EMF (App. A)
    ("ideal_diffusion_sign",
     "- cam * cap * (qBbR - qBbL)) / (cam + cap)",
     "+ cam * cap * (qBbR - qBbL)) / (cam + cap)", IDEAL_PINS),
    ("ideal_second_term_sign",
     "+ (cbm * vbR * qBaR + cbp * vbL * qBaL - cbm * cbp * (qBaR - qBaL)) / (cbm + cbp);",
     "- (cbm * vbR * qBaR + cbp * vbL * qBaL - cbm * cbp * (qBaR - qBaL)) / (cbm + cbp);", IDEAL_PINS),
    ("ideal_vbar_wrong_W",
     "double vL = alf * recL[1 + j] / WL, vR = alf * recR[1 + j] / WR;",
     "double vL = alf * recL[1 + j] / WL, vR = alf * recR[1 + j] / WL;", IDEAL_PINS),
    ("ideal_vhat_without_lapse",
     "vbar[d][j][c] = alp_at(X->alp, c) * prim[1 + j][c] / sqrt(1.0 + uu);",
     "vbar[d][j][c] = prim[1 + j][c] / sqrt(1.0 + uu);", IDEAL_PINS),
]


def test_every_mistake_applies_to_exactly_one_place():
    with open(SRC) as fh:
        src = fh.read()
    for name, old, new, *_ in MUTATIONS:
        assert src.count(old) == 1, name
        assert old != new, name


def _survives(case, tmpdir):
    """Compile the oracle with one planted mistake and run the pins against it;
    returns None when a pin fails, else the pins' output."""
    name, old, new = case[:3]
    pins = case[3] if len(case) > 3 else PINS
    with open(SRC) as fh:
        src = fh.read()
    mut = os.path.join(tmpdir, f"{name}.c")
    with open(mut, "w") as fh:
        fh.write(src.replace(old, new, 1))
    lib = os.path.join(tmpdir, f"lib{name}.so")
    oracle.compile_library(mut, lib)
    env = dict(os.environ, GRMHD_ORACLE_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins,
           *[f"--deselect={s}" for s in SKIP if pins is PINS]]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    # 1: some pin failed.  0 would be a mistake no pin sees; other codes are crashes or
    # collection errors, which do not count as being caught
    return None if r.returncode == 1 else f"rc {r.returncode}: " + r.stdout[-1500:] + r.stderr[-800:]


def test_every_planted_mistake_is_caught(tmp_path):
    """The cases run side by side (each in its own child process)."""
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        out = list(ex.map(lambda m: (m[0], _survives(m, str(tmp_path))), MUTATIONS))
    survivors = {name: msg for name, msg in out if msg is not None}
    assert not survivors, "\n\n".join(f"{k}: {v}" for k, v in survivors.items())
