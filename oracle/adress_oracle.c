/*
 * FP64 CPU oracle for one force-interpolation AdResS molecular-dynamics step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load this code; the product path never does.  It shares no
 * code, header, table generator or helper with the CUDA library.
 *
 * Every function is the plain definition, in double precision, in the order the
 * method states it:
 *   - resolution function lambda(R_alpha) of the molecule centre of mass, 1 in the
 *     AT region, 0 in the CG region, squared cosine through the hybrid layer
 *     (Sec. "Force interpolation"; Sec. "Potential energy interpolation" names the
 *     squared cosine);
 *   - force interpolation between molecules alpha and beta (Eq. 1):
 *       F_ab = l_a l_b F^AT_ab + (1 - l_a l_b) F^CG_ab,
 *     F^AT the sum of atom-atom forces, F^CG a COM-COM force (Sec. "Force
 *     interpolation");
 *   - intramolecular bonded terms, never interpolated (same section);
 *   - the thermodynamic force in the hybrid layer and its iterative construction from
 *     the density profile (Sec. "Free energy corrections and the thermodynamic force");
 *   - a Langevin thermostat (force interpolation needs thermostatting, Sec.
 *     "Potential energy interpolation") with velocity-Verlet integration.
 * Parity unpinned: the thermodynamic-force update rule (orc_tf_update) beyond its
 * identity and closed-form cases; the paper gives no formula for it.
 *
 * Built plainly (gcc -O2) every loop runs serially in the order written.  Built with
 * -fopenmp (the all-core CPU baseline), the per-atom and per-molecule loops run in
 * parallel and the linked-cell pair scan gives each thread its own force, energy and
 * per-molecule potential buffers, added in thread order afterwards: the same definition,
 * with floating-point sums in another order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "adress_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------------------
 * Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * published multipliers, key bumped by the published Weyl constants between rounds.
 * ------------------------------------------------------------------------------- */
void orc_philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k[2] = {key_in[0], key_in[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k[0] += W0;
      k[1] += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k[0];
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k[1];
    uint32_t n3 = (uint32_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  memcpy(out, c, sizeof(c));
}

/* Three uniforms in [0,1) for atom `gid` at time level `step`: two generator blocks with
 * counters (gid, step_lo, step_hi, 2 replica) and (gid, step_lo, step_hi, 2 replica + 1),
 * key (seed_lo, seed_hi); component d takes 32 high bits from the first block and 21 low
 * bits from the top of the second: u = (hi << 21 | lo >> 11) 2^-53. */
void orc_uniform3(uint64_t seed, int64_t replica, int64_t gid, int64_t step, double u[3]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t c0[4] = {(uint32_t)gid, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)(2 * replica)};
  uint32_t c1[4] = {(uint32_t)gid, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)(2 * replica + 1)};
  uint32_t hi[4], lo[4];
  orc_philox4x32(c0, key, hi);
  orc_philox4x32(c1, key, lo);
  for (int d = 0; d < 3; ++d)
    u[d] = (double)(((uint64_t)hi[d] << 21) | (lo[d] >> 11)) * (1.0 / 9007199254740992.0);
}

/* --------------------------------------------------------------------------------- */

static double minimg(double d, double L) { return d - L * nearbyint(d / L); }

double orc_weight(const orc_sys* s, double d) {
  /* lambda = 1 inside the AT half-width, squared cosine across the hybrid layer,
   * 0 beyond it; a zero-width layer is a step with no division. */
  if (d < s->d_at) return 1.0;
  if (d >= s->d_at + s->d_hy) return 0.0;
  double c = cos(0.5 * M_PI * (d - s->d_at) / s->d_hy);
  return c * c;
}

static double mol_mass(const orc_sys* s) {
  double m = 0;
  for (int k = 0; k < s->na; ++k) m += s->mass[k];
  return m;
}

/* Distance of a centre of mass to the nearest resolution centre (3D minimum image) and the
 * index of that centre (the first one on ties). */
static double nearest_center(const orc_sys* s, const double* R, int* kmin) {
  double best = INFINITY;
  int kb = 0;
  for (int k = 0; k < s->n_centers; ++k) {
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double t = minimg(R[d] - s->centers[3 * k + d], s->L[d]);
      r2 += t * t;
    }
    const double r = sqrt(r2);
    if (r < best) {
      best = r;
      kb = k;
    }
  }
  if (kmin) *kmin = kb;
  return best;
}

/* Centre of mass of every molecule (minimum-image unwrap relative to its first atom,
 * result wrapped into [0,L)), the distance d that the resolution function takes (slab: the
 * signed x-distance to the slab centre, so |d|; spheres: the non-negative distance to the
 * nearest centre) and lambda. */
void orc_com_lambda(const orc_sys* s, const double* x, double* R, double* dx_c, double* w) {
  const double Mt = mol_mass(s);
#pragma omp parallel for schedule(static)
  for (int a = 0; a < s->M; ++a) {
    const double* x0 = x + 3 * (size_t)a * s->na;
    double acc[3] = {0, 0, 0};
    for (int k = 0; k < s->na; ++k) {
      const double* xi = x0 + 3 * k;
      for (int d = 0; d < 3; ++d) acc[d] += s->mass[k] * (x0[d] + minimg(xi[d] - x0[d], s->L[d]));
    }
    for (int d = 0; d < 3; ++d) {
      double r = acc[d] / Mt;
      r -= s->L[d] * floor(r / s->L[d]);
      if (r >= s->L[d]) r -= s->L[d];
      R[3 * a + d] = r;
    }
    double dxc = s->n_centers > 0 ? nearest_center(s, R + 3 * a, NULL) : minimg(R[3 * a] - s->xc, s->L[0]);
    if (dx_c) dx_c[a] = dxc;
    if (w) w[a] = s->lam_uniform_on ? s->lam_uniform : orc_weight(s, fabs(dxc));
  }
}

/* --- pair potentials (force returned as F/r so that f_vec = (F/r) * r_vec) --------- */

static double wca_fr(const orc_sys* s, double r2, double* V) {
  double sr2 = s->sig * s->sig / r2;
  double sr6 = sr2 * sr2 * sr2;
  *V = 4.0 * s->eps * (sr6 * sr6 - sr6) + s->eps;
  return 24.0 * s->eps * (2.0 * sr6 * sr6 - sr6) / r2;
}

/* Atom pair (site i of one molecule, site j of another) of the water-like model:
 * Lennard-Jones with eps = sqrt(eps_i eps_j), sigma = (sigma_i + sigma_j)/2, potential
 * shifted so that V(rc) = 0, and reaction-field Coulomb
 * V = f q_i q_j (1/r + k_rf r^2 - c_rf), k_rf = (eps_rf - 1)/((2 eps_rf + 1) rc^3),
 * c_rf = 1/rc + k_rf rc^2 (so V(rc) = 0).  Returns F/r, sets V. */
static double ljrf_fr(const orc_sys* s, int si, int sj, double r2, double* V) {
  const double rc = s->rc_at;
  double fr = 0.0, v = 0.0;
  const double eps = sqrt(s->lj_eps[si] * s->lj_eps[sj]);
  if (eps > 0.0) {
    const double sg = 0.5 * (s->lj_sig[si] + s->lj_sig[sj]);
    const double sr2 = sg * sg / r2, sr6 = sr2 * sr2 * sr2;
    const double sc2 = sg * sg / (rc * rc), sc6 = sc2 * sc2 * sc2;
    v += 4.0 * eps * (sr6 * sr6 - sr6) - 4.0 * eps * (sc6 * sc6 - sc6);
    fr += 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
  }
  const double qq = s->coulomb_f * s->charge[si] * s->charge[sj];
  if (qq != 0.0) {
    const double krf = (s->eps_rf - 1.0) / ((2.0 * s->eps_rf + 1.0) * rc * rc * rc);
    const double crf = 1.0 / rc + krf * rc * rc;
    const double r = sqrt(r2);
    v += qq * (1.0 / r + krf * r2 - crf);
    fr += qq * (1.0 / (r2 * r) - 2.0 * krf);
  }
  *V = v;
  return fr;
}

/* Linear interpolation in the CG table: returns F(r) (positive = repulsive), sets V. */
static double cg_table(const orc_sys* s, double r, double* V) {
  double u = r / s->cg_dr;
  int k = (int)u;
  if (k >= s->cg_n) { *V = 0; return 0; }
  double t = u - k;
  *V = s->cgV[k] * (1.0 - t) + s->cgV[k + 1] * t;
  return s->cgF[k] * (1.0 - t) + s->cgF[k + 1] * t;
}

/* Thermodynamic force table, nodes d_k = k*tf_dx, linear interpolation, 0 outside. */
static double tf_table(const orc_sys* s, double d) {
  if (!s->tf || s->tf_n <= 0) return 0.0;
  double u = d / s->tf_dx;
  int k = (int)u;
  if (k + 1 < s->tf_n) {
    double t = u - k;
    return s->tf[k] * (1.0 - t) + s->tf[k + 1] * t;
  }
  if (k + 1 == s->tf_n && u == (double)k) return s->tf[k];
  return 0.0;
}

/* Accumulators: e[0]=E_AT (weighted), e[1]=E_CG (weighted), e[2]=E_bond,
 * e[3]=virial sum r.f (nonbonded + bonded). */

/* Interaction of molecules a and b (a != b), added to both (Newton's 3rd law): Eq. 1 with
 * w_ab = l_a l_b, or (energy interpolation) the pair terms of Eq. Hmix with
 * w_ab = (l_a + l_b)/2.  vat / vcg (may be NULL) collect the single-molecule potentials of
 * Eq. Hmix: half of every pair's unweighted AT and CG energy to each molecule. */
static void pair_ab(const orc_sys* s, const double* x, const double* R, const double* w, int a,
                    int b, double* f, double* e, double* vat, double* vcg, double sw) {
  const double wab = s->scheme == 1 ? 0.5 * (w[a] + w[b]) : w[a] * w[b];
  const int na = s->na;
  if (wab > 0.0) {
    const double rc2 = s->rc_at * s->rc_at;
    for (int i = a * na; i < (a + 1) * na; ++i)
      for (int j = b * na; j < (b + 1) * na; ++j) {
        double r[3], r2 = 0;
        for (int d = 0; d < 3; ++d) {
          r[d] = minimg(x[3 * i + d] - x[3 * j + d], s->L[d]);
          r2 += r[d] * r[d];
        }
        if (r2 >= rc2) continue;
        double V, fr = s->nb_model == 1 ? ljrf_fr(s, i - a * na, j - b * na, r2, &V) : wca_fr(s, r2, &V);
        for (int d = 0; d < 3; ++d) {
          f[3 * i + d] += wab * fr * r[d];
          f[3 * j + d] -= wab * fr * r[d];
        }
        e[0] += wab * V;
        e[3] += wab * fr * r2;
        if (vat) {
          vat[a] += 0.5 * V;
          vat[b] += 0.5 * V;
        }
      }
  }
  if (wab < 1.0) {
    double Rab[3], r2 = 0;
    for (int d = 0; d < 3; ++d) {
      Rab[d] = minimg(R[3 * a + d] - R[3 * b + d], s->L[d]);
      r2 += Rab[d] * Rab[d];
    }
    if (r2 < s->rc_cg * s->rc_cg) {
      double r = sqrt(r2), V = 0.0, F;
      if (s->mlp) {
        double feat[9];
        orc_pair_features(s, x, a, b, feat, NULL);
        orc_mlp_pair_force(s->mlp, 1, feat, &F);
      } else {
        F = cg_table(s, r, &V);
      }
      double c = (1.0 - wab) * F / r;
      const double cs = sw * c;  /* slow-force weight of multiple time stepping */
      const double Mt = mol_mass(s);
      /* the COM force reaches each atom in proportion m_i / M (dR/dx_i = m_i/M) */
      for (int k = 0; k < na; ++k)
        for (int d = 0; d < 3; ++d) {
          f[3 * (a * na + k) + d] += s->mass[k] / Mt * cs * Rab[d];
          f[3 * (b * na + k) + d] -= s->mass[k] / Mt * cs * Rab[d];
        }
      e[1] += (1.0 - wab) * V;
      if (vcg) {
        vcg[a] += 0.5 * V;
        vcg[b] += 0.5 * V;
      }
      e[3] += c * r2;
    }
  }
}

/* Harmonic angle (i, vertex j, k) of molecule a: V = k/2 (theta - theta0)^2 with
 * cos theta = u.v / (|u||v|), u = x_i - x_j, v = x_k - x_j.  F_i = -dV/dtheta dtheta/dx_i,
 * dtheta/dx_i = -(v/(|u||v|) - cos theta u/|u|^2) / sin theta; F_j = -(F_i + F_k). */
static void angle_mol(const orc_sys* s, const double* x, int a, double* f, double* e) {
  const int na = s->na;
  for (int q = 0; q < s->n_angles; ++q) {
    const int i = a * na + s->angles[3 * q], j = a * na + s->angles[3 * q + 1], k = a * na + s->angles[3 * q + 2];
    double u[3], v[3], uu = 0, vv = 0, uv = 0;
    for (int d = 0; d < 3; ++d) {
      u[d] = minimg(x[3 * i + d] - x[3 * j + d], s->L[d]);
      v[d] = minimg(x[3 * k + d] - x[3 * j + d], s->L[d]);
      uu += u[d] * u[d];
      vv += v[d] * v[d];
      uv += u[d] * v[d];
    }
    const double nu = sqrt(uu), nv = sqrt(vv);
    double c = uv / (nu * nv);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    const double th = acos(c), sn = sqrt(1.0 - c * c);
    const double dV = s->angle_k * (th - s->angle_theta0);
    e[2] += 0.5 * s->angle_k * (th - s->angle_theta0) * (th - s->angle_theta0);
    if (sn <= 0.0) continue;
    const double g = dV / sn;
    double fi[3], fk[3];
    for (int d = 0; d < 3; ++d) {
      fi[d] = g * (v[d] / (nu * nv) - c * u[d] / uu);
      fk[d] = g * (u[d] / (nu * nv) - c * v[d] / vv);
      f[3 * i + d] += fi[d];
      f[3 * k + d] += fk[d];
      f[3 * j + d] -= fi[d] + fk[d];
      e[3] += u[d] * fi[d] + v[d] * fk[d];
    }
  }
}

/* Bonded terms of molecule a, unweighted: FENE (+ optional WCA) or harmonic bonds on every
 * listed pair, and harmonic angles. */
static int bonded_mol(const orc_sys* s, const double* x, int a, double* f, double* e) {
  const int na = s->na;
  const double R02 = s->fene_r0 * s->fene_r0;
  if (s->n_angles > 0) angle_mol(s, x, a, f, e);
  for (int q = 0; q < s->nb; ++q) {
    int i = a * na + s->bonds[2 * q], j = a * na + s->bonds[2 * q + 1];
    double r[3], r2 = 0;
    for (int d = 0; d < 3; ++d) {
      r[d] = minimg(x[3 * i + d] - x[3 * j + d], s->L[d]);
      r2 += r[d] * r[d];
    }
    if (s->bond_model == 1) {
      /* harmonic: V = k/2 (r - r0)^2, F/r = -k (r - r0)/r */
      const double rr = sqrt(r2);
      const double fr = -s->bond_k * (rr - s->bond_r0) / rr;
      for (int d = 0; d < 3; ++d) {
        f[3 * i + d] += fr * r[d];
        f[3 * j + d] -= fr * r[d];
      }
      e[2] += 0.5 * s->bond_k * (rr - s->bond_r0) * (rr - s->bond_r0);
      e[3] += fr * r2;
      continue;
    }
    if (r2 >= R02) return ORC_ERR_BOND;
    double g = 1.0 - r2 / R02;
    double fr = -s->fene_k / g;
    double V = -0.5 * s->fene_k * R02 * log(g);
    if (s->intra_wca && r2 < s->rc_at * s->rc_at) {
      double Vw, frw = wca_fr(s, r2, &Vw);
      fr += frw;
      V += Vw;
    }
    for (int d = 0; d < 3; ++d) {
      f[3 * i + d] += fr * r[d];
      f[3 * j + d] -= fr * r[d];
    }
    e[2] += V;
    e[3] += fr * r2;
  }
  return ORC_OK;
}

/* Thermodynamic force on hybrid-layer molecules, away from the AT region when positive
 * (slab: along x; spheres: along the direction from the nearest centre), spread over the
 * atoms by mass fraction. */
static void tf_forces(const orc_sys* s, const double* R, const double* dxc, double* f, double sw) {
  if (s->lam_uniform_on) return;
  const double Mt = mol_mass(s);
  for (int a = 0; a < s->M; ++a) {
    double d = fabs(dxc[a]);
    if (d < s->d_at || d >= s->d_at + s->d_hy) continue;
    double dir[3] = {dxc[a] < 0 ? -1.0 : 1.0, 0.0, 0.0};
    if (s->n_centers > 0) {
      int kc;
      nearest_center(s, R + 3 * a, &kc);
      for (int q = 0; q < 3; ++q) dir[q] = minimg(R[3 * a + q] - s->centers[3 * kc + q], s->L[q]) / d;
    }
    const double F = sw * tf_table(s, d);
    for (int k = 0; k < s->na; ++k)
      for (int q = 0; q < 3; ++q) f[3 * (a * s->na + k) + q] += s->mass[k] / Mt * F * dir[q];
  }
}

/* Free-energy correction derivative g(l) = dDF/dl: linear between the nodes l_k = k/(n-1). */
double orc_fec_g(const orc_sys* s, double l) {
  if (s->fec_n < 2) return 0.0;
  const double u = l * (s->fec_n - 1);
  int k = (int)floor(u);
  if (k >= s->fec_n - 1) return s->fec[s->fec_n - 1];
  if (k < 0) k = 0;
  const double t = u - k;
  return s->fec[k] * (1.0 - t) + s->fec[k + 1] * t;
}

/* Drift force of energy interpolation (Eq. Hmix): the position derivative of l(R_a) in
 * l_a V_AT_a + (1 - l_a) V_CG_a gives F_i = -(V_AT_a - V_CG_a) l'(d_a) (m_i/M) grad d_a on
 * the atoms of molecule a, with l'(d) = -(pi/(2 d_hy)) sin(pi (d - d_at)/d_hy) in the hybrid
 * layer and 0 elsewhere, grad d = sign(x - x_c) x (slab) or (R - c)/d (nearest centre).
 * The free-energy correction -DF(l_a) adds +g(l_a) l'(d_a) grad d_a.  vat == NULL (lambda
 * held fixed) gives neither. */
static void drift_forces(const orc_sys* s, const double* R, const double* dxc, const double* w,
                         const double* vat, const double* vcg, double* f, double sw) {
  if (!vat || s->d_hy <= 0.0 || s->lam_uniform_on) return;
  const double Mt = mol_mass(s);
  for (int a = 0; a < s->M; ++a) {
    const double d = fabs(dxc[a]);
    if (d <= s->d_at || d >= s->d_at + s->d_hy) continue;
    const double dl = -(M_PI / (2.0 * s->d_hy)) * sin(M_PI * (d - s->d_at) / s->d_hy);
    double dir[3] = {dxc[a] < 0 ? -1.0 : 1.0, 0.0, 0.0};
    if (s->n_centers > 0) {
      int kc;
      nearest_center(s, R + 3 * a, &kc);
      for (int q = 0; q < 3; ++q) dir[q] = minimg(R[3 * a + q] - s->centers[3 * kc + q], s->L[q]) / d;
    }
    /* fast part -V_AT l', slow part +(V_CG + g) l' (weighted by sw) */
    const double F = -(vat[a] - sw * (vcg[a] + orc_fec_g(s, w[a]))) * dl;
    for (int k = 0; k < s->na; ++k)
      for (int q = 0; q < 3; ++q) f[3 * (a * s->na + k) + q] += s->mass[k] / Mt * F * dir[q];
  }
}

/* Largest atom-to-COM distance over all molecules. */
static double max_extent(const orc_sys* s, const double* x, const double* R) {
  double m = 0;
  for (int a = 0; a < s->M; ++a)
    for (int k = 0; k < s->na; ++k) {
      double r2 = 0;
      for (int d = 0; d < 3; ++d) {
        double t = minimg(x[3 * (a * s->na + k) + d] - R[3 * a + d], s->L[d]);
        r2 += t * t;
      }
      if (r2 > m) m = r2;
    }
  return sqrt(m);
}

/* Every pair (a, b > a) of molecule a with the molecules of its cell and the 26 cells around
 * it (each distinct cell once, so that a box of two cells along an axis counts no pair
 * twice). */
static void cell_scan(const orc_sys* s, const double* x, const double* R, const double* w, int a, const int nc[3],
                      const int* cell, const int* head, const int* next, double* f, double* acc, double* vat,
                      double* vcg, double sw) {
  int c = cell[a];
  int cz = c % nc[2], cy = (c / nc[2]) % nc[1], cx = c / (nc[1] * nc[2]);
  int seen[27], ns = 0;
  for (int ox = -1; ox <= 1; ++ox)
    for (int oy = -1; oy <= 1; ++oy)
      for (int oz = -1; oz <= 1; ++oz) {
        int nx = ((cx + ox) % nc[0] + nc[0]) % nc[0];
        int ny = ((cy + oy) % nc[1] + nc[1]) % nc[1];
        int nz = ((cz + oz) % nc[2] + nc[2]) % nc[2];
        int nbc = (nx * nc[1] + ny) * nc[2] + nz, dup = 0;
        for (int q = 0; q < ns; ++q) dup |= (seen[q] == nbc);
        if (dup) continue;
        seen[ns++] = nbc;
        for (int b = head[nbc]; b >= 0; b = next[b])
          if (b > a) pair_ab(s, x, R, w, a, b, f, acc, vat, vcg, sw);
      }
}

/* Conservative forces (no thermostat).  method 0: every molecule pair a<b;
 * method 1: a linked-cell scan over COM cells no smaller than the largest pair reach.
 * w_override (may be NULL) replaces lambda for every molecule. */
/* Forces with the slow (CG) part weighted by sw: 1 for the plain force; with multiple time
 * stepping n at outer steps and 0 in between (energies and virial stay unweighted). */
static int forces_sw(const orc_sys* s, const double* x, int method, const double* w_override, double* f,
                     double* e, double sw) {
  const int M = s->M;
  double* R = (double*)malloc(sizeof(double) * 3 * M);
  double* dxc = (double*)malloc(sizeof(double) * M);
  double* w = (double*)malloc(sizeof(double) * M);
  orc_com_lambda(s, x, R, dxc, w);
  if (w_override) memcpy(w, w_override, sizeof(double) * M);
  memset(f, 0, sizeof(double) * 3 * (size_t)M * s->na);
  double acc[4] = {0, 0, 0, 0};
  int st = ORC_OK;
  double* vat = s->scheme == 1 ? (double*)calloc(M, sizeof(double)) : NULL;
  double* vcg = s->scheme == 1 ? (double*)calloc(M, sizeof(double)) : NULL;

  if (method == 0) {
    for (int a = 0; a < M; ++a)
      for (int b = a + 1; b < M; ++b) pair_ab(s, x, R, w, a, b, f, acc, vat, vcg, sw);
  } else {
    double ext = max_extent(s, x, R);
    double reach = s->rc_cg > s->rc_at + 2 * ext ? s->rc_cg : s->rc_at + 2 * ext;
    int nc[3];
    for (int d = 0; d < 3; ++d) {
      nc[d] = (int)floor(s->L[d] / reach);
      if (nc[d] < 1) nc[d] = 1;
    }
    int ncell = nc[0] * nc[1] * nc[2];
    int* head = (int*)malloc(sizeof(int) * ncell);
    int* next = (int*)malloc(sizeof(int) * M);
    int* cell = (int*)malloc(sizeof(int) * M);
    for (int c = 0; c < ncell; ++c) head[c] = -1;
    for (int a = M - 1; a >= 0; --a) {
      int ci[3];
      for (int d = 0; d < 3; ++d) {
        ci[d] = (int)(R[3 * a + d] / s->L[d] * nc[d]);
        if (ci[d] >= nc[d]) ci[d] = nc[d] - 1;
      }
      cell[a] = (ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
      next[a] = head[cell[a]];
      head[cell[a]] = a;
    }
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    if (nt == 1) {
      for (int a = 0; a < M; ++a) cell_scan(s, x, R, w, a, nc, cell, head, next, f, acc, vat, vcg, sw);
    } else {
      /* all-core build: private buffers per thread, added in thread order */
      const size_t n3 = (size_t)3 * M * s->na;
      double* fb = (double*)calloc((size_t)nt * n3, sizeof(double));
      double* eb = (double*)calloc((size_t)nt * 4, sizeof(double));
      double* vb = vat ? (double*)calloc((size_t)nt * 2 * M, sizeof(double)) : NULL;
#pragma omp parallel num_threads(nt)
      {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double* vt = vb ? vb + (size_t)t * 2 * M : NULL;
#pragma omp for schedule(static)
        for (int a = 0; a < M; ++a)
          cell_scan(s, x, R, w, a, nc, cell, head, next, fb + (size_t)t * n3, eb + 4 * t, vt, vt ? vt + M : NULL, sw);
      }
      for (int t = 0; t < nt; ++t) {
        for (size_t i = 0; i < n3; ++i) f[i] += fb[(size_t)t * n3 + i];
        for (int k = 0; k < 4; ++k) acc[k] += eb[4 * t + k];
        if (vb)
          for (int a = 0; a < M; ++a) {
            vat[a] += vb[(size_t)t * 2 * M + a];
            vcg[a] += vb[(size_t)t * 2 * M + M + a];
          }
      }
      free(fb); free(eb); free(vb);
    }
    free(head); free(next); free(cell);
  }
  for (int a = 0; a < M && st == ORC_OK; ++a) st = bonded_mol(s, x, a, f, acc);
  tf_forces(s, R, dxc, f, sw);
  if (vat) {
    drift_forces(s, R, dxc, w, w_override ? NULL : vat, vcg, f, sw);
    free(vat);
    free(vcg);
  }
  if (e) memcpy(e, acc, sizeof(acc));
  free(R); free(dxc); free(w);
  return st;
}

/* Langevin friction and noise for atom gid at time level `step`:
 *   F_L = -gamma m v + sqrt(24 gamma kT m / dt) (u - 1/2),
 * u uniform in [0,1) from orc_uniform3 (Philox4x32-10). */
static void langevin(const orc_sys* s, const double* v, int64_t step, double* f) {
  const int N = s->M * s->na;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i) {
    double m = s->mass[i % s->na];
    double amp = sqrt(24.0 * s->gamma * s->kT * m / s->dt);
    double u[3];
    orc_uniform3(s->seed, s->replica, i, step, u);
    for (int d = 0; d < 3; ++d) f[3 * i + d] += -s->gamma * m * v[3 * i + d] + amp * (u[d] - 0.5);
  }
}

/* Velocity Verlet with the thermostat force evaluated with the half-step velocity:
 *   v += dt/2 f/m;  x += dt v;  wrap;  f = F(x) + F_L(v; step+1);  v += dt/2 f/m.
 * (x, v, f) hold time level `step0` on entry and step0+nsteps on return. */
/* Slow-force weight at time level `step`: multiple time stepping (Sec. "Multiple time
 * stepping in adaptive resolution simulations", impulse r-RESPA) applies the CG forces as an
 * impulse of n inner steps at every n-th time level and not in between. */
static double slow_weight(const orc_sys* s, int64_t step) {
  if (s->respa_n <= 1) return 1.0;
  return step % s->respa_n == 0 ? (double)s->respa_n : 0.0;
}

int orc_forces(const orc_sys* s, const double* x, int method, const double* w_override, double* f,
               double* e) {
  return forces_sw(s, x, method, w_override, f, e, 1.0);
}

int orc_forces_step(const orc_sys* s, const double* x, int64_t step, double* f, double* e) {
  return forces_sw(s, x, 1, NULL, f, e, slow_weight(s, step));
}

int orc_run(const orc_sys* s, double* x, double* v, double* f, int64_t step0, int nsteps, int method) {
  const int N = s->M * s->na;
  for (int n = 0; n < nsteps; ++n) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
      double m = s->mass[i % s->na];
      for (int d = 0; d < 3; ++d) {
        v[3 * i + d] += 0.5 * s->dt * f[3 * i + d] / m;
        double y = x[3 * i + d] + s->dt * v[3 * i + d];
        if (y < 0) y += s->L[d];
        if (y >= s->L[d]) y -= s->L[d];
        x[3 * i + d] = y;
      }
    }
    int st = forces_sw(s, x, method, NULL, f, NULL, slow_weight(s, step0 + n + 1));
    if (st != ORC_OK) return st;
    if (s->gamma != 0.0) langevin(s, v, step0 + n + 1, f);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
      double m = s->mass[i % s->na];
      for (int d = 0; d < 3; ++d) v[3 * i + d] += 0.5 * s->dt * f[3 * i + d] / m;
    }
  }
  return ORC_OK;
}

/* Thermostat force alone (for tests): f += F_L(v; step). */
void orc_langevin_force(const orc_sys* s, const double* v, int64_t step, double* f) {
  langevin(s, v, step, f);
}

/* Kinetic energy and total momentum: out = {KE, Px, Py, Pz}. */
void orc_kinetic(const orc_sys* s, const double* v, double* out) {
  const int N = s->M * s->na;
  double ke = 0, p[3] = {0, 0, 0};
  for (int i = 0; i < N; ++i) {
    double m = s->mass[i % s->na];
    for (int d = 0; d < 3; ++d) {
      ke += 0.5 * m * v[3 * i + d] * v[3 * i + d];
      p[d] += m * v[3 * i + d];
    }
  }
  out[0] = ke; out[1] = p[0]; out[2] = p[1]; out[3] = p[2];
}

/* COM density histograms: counts_d[k] over |x_com - xc| in bins of tf_dx (folded about
 * the centre, nd bins), counts_x[k] over x_com in bins of Lx/nx.  Counts are added. */
void orc_density(const orc_sys* s, const double* x, int nd, int64_t* counts_d, int nx,
                 int64_t* counts_x) {
  double* R = (double*)malloc(sizeof(double) * 3 * s->M);
  double* dxc = (double*)malloc(sizeof(double) * s->M);
  orc_com_lambda(s, x, R, dxc, NULL);
  for (int a = 0; a < s->M; ++a) {
    int kd = (int)floor(fabs(dxc[a]) / s->tf_dx);
    if (counts_d && kd < nd) counts_d[kd] += 1;
    int kx = (int)floor(R[3 * a] / s->L[0] * nx);
    if (kx >= nx) kx = nx - 1;
    if (counts_x) counts_x[kx] += 1;
  }
  free(R); free(dxc);
}

/* COM pair-distance histogram (the numerator of the radial distribution function g(r),
 * the structural observable that judges a coarse-grained model): counts[k] += number of
 * molecule pairs a < b whose minimum-image COM distance r has floor(r / dr) = k < nbins.
 * All pairs, no lists. */
void orc_rdf(const orc_sys* s, const double* x, int nbins, double dr, int64_t* counts) {
  double* R = (double*)malloc(sizeof(double) * 3 * s->M);
  orc_com_lambda(s, x, R, NULL, NULL);
  for (int a = 0; a < s->M; ++a)
    for (int b = a + 1; b < s->M; ++b) {
      double r2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        double t = minimg(R[3 * a + d] - R[3 * b + d], s->L[d]);
        r2 += t * t;
      }
      int k = (int)floor(sqrt(r2) / dr);
      if (k < nbins) counts[k] += 1;
    }
  free(R);
}

/* Thermodynamic-force iteration: tf_k <- tf_k - alpha * g_k for hybrid-layer nodes,
 * where rho_k = counts_d[k] / (nsamples * V_k) is the folded COM density in
 * bin [k dx, (k+1) dx) (V_k: two slabs 2 dx Ly Lz, or n_centers spherical shells),
 * g_k = (rho_k - rho_{k-1}) / dx is its gradient at node d_k
 * (g_0 = 0 by symmetry, g at the last node one-sided), smoothed by a three-point moving
 * average.  Parity unpinned beyond zero-gradient and linear-profile cases. */
void orc_tf_update(const orc_sys* s, double* tf, int n, const int64_t* counts_d, int nd,
                   double nsamples, double alpha) {
  double* rho = (double*)calloc(n + 1, sizeof(double));
  double* g = (double*)calloc(n, sizeof(double));
  const double dx = s->tf_dx;
  for (int k = 0; k < n && k < nd; ++k) {
    /* bin volume: two slabs of width dx, or a spherical shell around each centre (exact
     * when the spheres do not overlap) */
    const double vol = s->n_centers > 0
                           ? nsamples * s->n_centers * 4.0 / 3.0 * M_PI * ((k + 1.0) * (k + 1.0) * (k + 1.0) - (double)k * k * k) * dx * dx * dx
                           : nsamples * 2.0 * dx * s->L[1] * s->L[2];
    rho[k] = counts_d[k] / vol;
  }
  for (int k = 1; k < n; ++k) g[k] = (k < nd ? (rho[k] - rho[k - 1]) : 0.0) / s->tf_dx;
  for (int k = 0; k < n; ++k) {
    double sum = 0;
    int cnt = 0;
    for (int q = k - 1; q <= k + 1; ++q)
      if (q >= 0 && q < n) { sum += g[q]; ++cnt; }
    double dk = k * s->tf_dx;
    if (dk >= s->d_at && dk <= s->d_at + s->d_hy) tf[k] -= alpha * sum / cnt;
  }
  free(rho); free(g);
}

/* =================================================================================
 * Learned coarse-grained pair force (force matching).  The paper's CG force is "a CG
 * force between the molecules, typically evaluated between their centers of mass"
 * (Sec. "Force interpolation"); the learned variant replaces the tabulated F^CG by a
 * small network of the COM distance and orientation invariants, trained so that its
 * output matches the atomistic force between the two molecules projected on the COM axis.
 *
 * Features of a molecule pair (a, b):  e = minimg(R_b - R_a)/d, d = |minimg(R_b - R_a)|;
 *   s_a = the na projections (x_i - R_a).e of a's atoms, sorted ascending;
 *   s_b = the na projections (x_j - R_b).(-e) of b's atoms, sorted ascending;
 *   feature vector (d, s_a[0..3], s_b[0..3]) (padded with 0 when na < 4).
 * Target: t = (sum_{i in a, j in b} f^WCA_ij) . (-e), the atomistic force on a from b along
 * the COM axis (positive = repulsive).
 * Network: x = (feat - mean)/std; z1 = W1 x + b1; h1 = silu(z1); z2 = W2 h1 + b2;
 *   h2 = silu(z2); y = w3.h2 + b3; force = out_scale * y.  With bf16 != 0 the inputs, W1,
 *   W2 and h1 are rounded to bfloat16 (round to nearest even) before their products, as the
 *   tensor-core path stores them.  Pair force used in dynamics: the mean of the network on
 *   (d, s_a, s_b) and on (d, s_b, s_a), so both molecules of a pair see the same value.
 * ================================================================================= */

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double dsilu(double z) {
  double sg = 1.0 / (1.0 + exp(-z));
  return sg * (1.0 + z * (1.0 - sg));
}

double orc_bf16(double v) {
  float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return v; /* inf / nan unchanged */
  uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);     /* round to nearest even */
  r &= 0xffff0000u;
  memcpy(&f, &r, 4);
  return (double)f;
}

static void sort4(double* v, int n) {
  for (int i = 1; i < n; ++i) {
    double key = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > key) {
      v[j + 1] = v[j];
      --j;
    }
    v[j + 1] = key;
  }
}

/* Features and target of the pair (a, b) at positions x. */
void orc_pair_features(const orc_sys* s, const double* x, int a, int b, double* feat, double* target) {
  double R[2][3];
  const int mol[2] = {a, b};
  const double Mt = mol_mass(s);
  for (int q = 0; q < 2; ++q) {
    const double* x0 = x + 3 * (size_t)mol[q] * s->na;
    for (int d = 0; d < 3; ++d) {
      double acc = 0;
      for (int k = 0; k < s->na; ++k) acc += s->mass[k] * (x0[d] + minimg(x0[3 * k + d] - x0[d], s->L[d]));
      R[q][d] = acc / Mt;
    }
  }
  double e[3], dd = 0;
  for (int d = 0; d < 3; ++d) {
    e[d] = minimg(R[1][d] - R[0][d], s->L[d]);
    dd += e[d] * e[d];
  }
  dd = sqrt(dd);
  for (int d = 0; d < 3; ++d) e[d] /= dd;
  double sa[4] = {0, 0, 0, 0}, sb[4] = {0, 0, 0, 0};
  for (int k = 0; k < s->na; ++k) {
    double pa = 0, pb = 0;
    for (int d = 0; d < 3; ++d) {
      pa += minimg(x[3 * ((size_t)a * s->na + k) + d] - R[0][d], s->L[d]) * e[d];
      pb -= minimg(x[3 * ((size_t)b * s->na + k) + d] - R[1][d], s->L[d]) * e[d];
    }
    sa[k] = pa;
    sb[k] = pb;
  }
  sort4(sa, s->na);
  sort4(sb, s->na);
  feat[0] = dd;
  for (int k = 0; k < 4; ++k) {
    feat[1 + k] = sa[k];
    feat[5 + k] = sb[k];
  }
  if (target) {
    double F[3] = {0, 0, 0};
    const double rc2 = s->rc_at * s->rc_at;
    for (int i = a * s->na; i < (a + 1) * s->na; ++i)
      for (int j = b * s->na; j < (b + 1) * s->na; ++j) {
        double r[3], r2 = 0;
        for (int d = 0; d < 3; ++d) {
          r[d] = minimg(x[3 * i + d] - x[3 * j + d], s->L[d]);
          r2 += r[d] * r[d];
        }
        if (r2 >= rc2) continue;
        double V, fr = s->nb_model == 1 ? ljrf_fr(s, i - a * s->na, j - b * s->na, r2, &V) : wca_fr(s, r2, &V);
        for (int d = 0; d < 3; ++d) F[d] += fr * r[d];
      }
    *target = -(F[0] * e[0] + F[1] * e[1] + F[2] * e[2]);
  }
}

/* All pairs a < b whose COM distance is below rc: features [n][9], targets [n], ids [n][2].
 * Returns the number of pairs written (at most cap; the count of all pairs if larger). */
long orc_collect_pairs(const orc_sys* s, const double* x, double rc, long cap, double* feat, double* target,
                       int* ids) {
  double* R = (double*)malloc(sizeof(double) * 3 * s->M);
  orc_com_lambda(s, x, R, NULL, NULL);
  long n = 0;
  for (int a = 0; a < s->M; ++a)
    for (int b = a + 1; b < s->M; ++b) {
      double r2 = 0;
      for (int d = 0; d < 3; ++d) {
        double t = minimg(R[3 * b + d] - R[3 * a + d], s->L[d]);
        r2 += t * t;
      }
      if (r2 >= rc * rc) continue;
      if (n < cap) {
        orc_pair_features(s, x, a, b, feat + 9 * n, target + n);
        ids[2 * n] = a;
        ids[2 * n + 1] = b;
      }
      ++n;
    }
  free(R);
  return n;
}


/* Network output y (before out_scale) for one feature vector; keeps z1, h1, z2, h2 when
 * cache != NULL (cache = [4][nh]). */
static double mlp_forward1(const orc_mlp* m, const double* feat, double* cache) {
  const int nh = m->nh;
  double x[9], z1[256], h1[256], z2[256], h2[256];
  for (int k = 0; k < 9; ++k) {
    x[k] = (feat[k] - m->in_mean[k]) / m->in_std[k];
    if (m->bf16) x[k] = orc_bf16(x[k]);
  }
  for (int o = 0; o < nh; ++o) {
    double acc = m->b1[o];
    for (int k = 0; k < 9; ++k) acc += (m->bf16 ? orc_bf16(m->W1[o * 9 + k]) : m->W1[o * 9 + k]) * x[k];
    z1[o] = acc;
    h1[o] = silu(acc);
    if (m->bf16) h1[o] = orc_bf16(h1[o]);
  }
  for (int o = 0; o < nh; ++o) {
    double acc = m->b2[o];
    for (int k = 0; k < nh; ++k) acc += (m->bf16 ? orc_bf16(m->W2[o * nh + k]) : m->W2[o * nh + k]) * h1[k];
    z2[o] = acc;
    h2[o] = silu(acc);
  }
  double y = m->b3;
  for (int k = 0; k < nh; ++k) y += m->w3[k] * h2[k];
  if (cache) {
    memcpy(cache, z1, sizeof(double) * nh);
    memcpy(cache + nh, h1, sizeof(double) * nh);
    memcpy(cache + 2 * nh, z2, sizeof(double) * nh);
    memcpy(cache + 3 * nh, h2, sizeof(double) * nh);
  }
  return y;
}

/* Forward over n feature vectors: y [n] (network output, before out_scale). */
void orc_mlp_forward(const orc_mlp* m, long n, const double* feat, double* y) {
  for (long s = 0; s < n; ++s) y[s] = mlp_forward1(m, feat + 9 * s, NULL);
}

/* Symmetrised pair force (after out_scale) for n feature vectors. */
void orc_mlp_pair_force(const orc_mlp* m, long n, const double* feat, double* f) {
  for (long s = 0; s < n; ++s) {
    double sw[9];
    sw[0] = feat[9 * s];
    for (int k = 0; k < 4; ++k) {
      sw[1 + k] = feat[9 * s + 5 + k];
      sw[5 + k] = feat[9 * s + 1 + k];
    }
    f[s] = 0.5 * m->out_scale * (mlp_forward1(m, feat + 9 * s, NULL) + mlp_forward1(m, sw, NULL));
  }
}

/* Loss L = (1/n) sum_s (y_s - t_s/out_scale)^2 and its gradient with respect to every
 * parameter (gW1 [nh][9], gb1, gW2 [nh][nh], gb2, gw3, gb3), by the chain rule through the
 * layers above (rounding to bfloat16 treated as the identity). Returns L. */
double orc_mlp_loss_grad(const orc_mlp* m, long n, const double* feat, const double* target, double* gW1,
                         double* gb1, double* gW2, double* gb2, double* gw3, double* gb3) {
  const int nh = m->nh;
  memset(gW1, 0, sizeof(double) * nh * 9);
  memset(gb1, 0, sizeof(double) * nh);
  memset(gW2, 0, sizeof(double) * nh * nh);
  memset(gb2, 0, sizeof(double) * nh);
  memset(gw3, 0, sizeof(double) * nh);
  *gb3 = 0;
  double loss = 0;
  double cache[4 * 256], x[9], d2[256], d1[256];
  for (long s = 0; s < n; ++s) {
    const double* f = feat + 9 * s;
    double y = mlp_forward1(m, f, cache);
    double r = y - target[s] / m->out_scale;
    loss += r * r;
    double dy = 2.0 * r / n;
    const double *z1 = cache, *h1 = cache + nh, *z2 = cache + 2 * nh, *h2 = cache + 3 * nh;
    for (int k = 0; k < 9; ++k) {
      x[k] = (f[k] - m->in_mean[k]) / m->in_std[k];
      if (m->bf16) x[k] = orc_bf16(x[k]);
    }
    *gb3 += dy;
    for (int k = 0; k < nh; ++k) {
      gw3[k] += dy * h2[k];
      d2[k] = dy * m->w3[k] * dsilu(z2[k]);
      gb2[k] += d2[k];
    }
    for (int o = 0; o < nh; ++o)
      for (int k = 0; k < nh; ++k) gW2[o * nh + k] += d2[o] * h1[k];
    for (int k = 0; k < nh; ++k) {
      double acc = 0;
      for (int o = 0; o < nh; ++o) acc += d2[o] * (m->bf16 ? orc_bf16(m->W2[o * nh + k]) : m->W2[o * nh + k]);
      d1[k] = acc * dsilu(z1[k]);
      gb1[k] += d1[k];
    }
    for (int o = 0; o < nh; ++o)
      for (int k = 0; k < 9; ++k) gW1[o * 9 + k] += d1[o] * x[k];
  }
  return loss / n;
}
