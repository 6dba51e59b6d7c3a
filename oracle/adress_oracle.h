/*
 * FP64 CPU oracle for force-interpolation AdResS (test infrastructure only; see
 * adress_oracle.c).  Positions, velocities and forces are (N, 3) row-major doubles,
 * atoms of molecule a at a*na .. a*na+na-1.
 */
#ifndef ADRESS_ORACLE_H
#define ADRESS_ORACLE_H
#include <stdint.h>

enum { ORC_OK = 0, ORC_ERR_BOND = 1 };

/* learned CG pair force (force matching) */
typedef struct {
  int nh;
  const double *W1, *b1, *W2, *b2, *w3;
  double b3;
  const double *in_mean, *in_std;
  double out_scale;
  int bf16;
} orc_mlp;

typedef struct {
  int M, na;
  const double* mass; /* na per-site masses */
  double L[3];
  double xc, d_at, d_hy; /* slab centre, AT half-width, hybrid width */
  double eps, sig, rc_at; /* WCA between atoms of different molecules */
  int nb;
  const int* bonds; /* 2*nb local atom indices */
  double fene_k, fene_r0;
  int intra_wca;
  const double *cgF, *cgV; /* CG table, cg_n+1 nodes at k*cg_dr */
  int cg_n;
  double cg_dr, rc_cg;
  const double* tf; /* thermodynamic force, tf_n nodes at k*tf_dx */
  int tf_n;
  double tf_dx;
  double kT, gamma, dt;
  uint64_t seed;
  int64_t replica;
  const orc_mlp* mlp; /* when non-NULL the CG force of Eq. 1 is the learned pair force */
  /* water-like molecules (nb_model 1): between atoms of different molecules, Lennard-Jones
   * with Lorentz-Berthelot site pairs, shifted to zero at rc_at, plus reaction-field
   * Coulomb; bond_model 1: harmonic bonds on the listed pairs; harmonic angles */
  int nb_model;
  const double *charge, *lj_eps, *lj_sig; /* na each */
  double coulomb_f, eps_rf;
  int bond_model;
  double bond_k, bond_r0;
  int n_angles;
  const int* angles; /* 3 * n_angles local indices (i, vertex, k) */
  double angle_k, angle_theta0;
  /* self-adjusting geometry (Sec. "Self-adjusting adaptive resolution simulations"): with
   * n_centers > 0 the AT region is the union of spheres of radius d_at around the centres,
   * d is the distance of the COM to the nearest centre (3D minimum image) and the
   * thermodynamic force acts along the direction from that centre */
  int n_centers;
  const double* centers; /* 3 * n_centers */
  /* scheme 0: force interpolation (Eq. 1); scheme 1: energy interpolation (Eq. Hmix,
   * H-AdResS): pair terms weighted by (l_a + l_b)/2 and the drift force
   * -(V_AT_a - V_CG_a) grad l_a on the atoms of each hybrid molecule */
  int scheme;
  /* free-energy correction of energy interpolation (Sec. "Free energy corrections and the
   * thermodynamic force"): g(l) = dDF/dl per molecule at fec_n >= 2 equidistant nodes on
   * [0, 1], linear in between; H gains -sum_a DF(l_a), DF(l) = int_0^l g.  fec_n = 0: none */
  int fec_n;
  const double* fec;
  /* Kirkwood thermodynamic integration: lam_uniform_on != 0 gives every molecule
   * l = lam_uniform (no position dependence, hence no thermodynamic or drift force) */
  int lam_uniform_on;
  double lam_uniform;
  /* multiple time stepping (impulse r-RESPA): respa_n > 1 applies the slow forces (CG pair
   * forces, thermodynamic force, the CG part of the drift force and the free-energy
   * correction) as n dt impulses at time levels divisible by n; dt is the inner step */
  int respa_n;
} orc_sys;

void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_uniform3(uint64_t seed, int64_t replica, int64_t gid, int64_t step, double u[3]);
double orc_weight(const orc_sys* s, double d);
double orc_fec_g(const orc_sys* s, double l);
void orc_com_lambda(const orc_sys* s, const double* x, double* R, double* dx_c, double* w);
int orc_forces(const orc_sys* s, const double* x, int method, const double* w_override, double* f,
               double* e);
int orc_run(const orc_sys* s, double* x, double* v, double* f, int64_t step0, int nsteps, int method);
int orc_forces_step(const orc_sys* s, const double* x, int64_t step, double* f, double* e);
void orc_langevin_force(const orc_sys* s, const double* v, int64_t step, double* f);
void orc_kinetic(const orc_sys* s, const double* v, double* out);
void orc_density(const orc_sys* s, const double* x, int nd, int64_t* counts_d, int nx,
                 int64_t* counts_x);
void orc_tf_update(const orc_sys* s, double* tf, int n, const int64_t* counts_d, int nd,
                   double nsamples, double alpha);
void orc_rdf(const orc_sys* s, const double* x, int nbins, double dr, int64_t* counts);

double orc_bf16(double v);
void orc_pair_features(const orc_sys* s, const double* x, int a, int b, double* feat, double* target);
long orc_collect_pairs(const orc_sys* s, const double* x, double rc, long cap, double* feat, double* target,
                       int* ids);
void orc_mlp_forward(const orc_mlp* m, long n, const double* feat, double* y);
void orc_mlp_pair_force(const orc_mlp* m, long n, const double* feat, double* f);
double orc_mlp_loss_grad(const orc_mlp* m, long n, const double* feat, const double* target, double* gW1,
                         double* gb1, double* gW2, double* gb2, double* gw3, double* gb3);
#endif
