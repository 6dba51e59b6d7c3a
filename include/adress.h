/*
 * adress.h — C ABI of the GB300 (sm_103a) AdResS step.
 *
 * One AdResS molecular-dynamics step of the paper's force-interpolation scheme
 * (ESPResSo++ 2.0, Sec. "Force interpolation", Eq. 1):
 *   F_ab = l(R_a) l(R_b) F^AT_ab + (1 - l(R_a) l(R_b)) F^CG_ab,
 * where l is the resolution function of the molecule centre of mass R (1 in the
 * atomistic region, 0 in the coarse-grained region, squared cosine across the hybrid
 * layer), F^AT the sum of atom-atom forces between the two molecules and F^CG a
 * COM-COM force.  Intramolecular bonds are not interpolated (same section); a
 * thermodynamic force acts in the hybrid layer (Sec. "Free energy corrections and the
 * thermodynamic force"); force interpolation needs a thermostat (Sec. "Potential energy
 * interpolation"), here Langevin inside velocity Verlet.  The configuration also selects
 * energy interpolation (H-AdResS, Eq. Hmix, with its drift force, a free-energy
 * correction and Kirkwood integration for it), a self-adjusting AT region around moving
 * centres, and multiple time stepping of the CG forces; see adress_config.
 *
 * Conventions for every call:
 *  - All state arrays are caller-owned DEVICE memory in structure-of-arrays layout
 *    [3][N] (x components of all atoms, then y, then z); atoms of molecule a are
 *    a*na .. a*na+na-1.  The library never frees caller memory.
 *  - The handle owns its lists, tables, scratch buffers and CUDA graphs; it allocates
 *    them with cudaMalloc in adress_init / adress_build_lists and frees them in
 *    adress_destroy.
 *  - Work is enqueued on the stream given to adress_init and runs asynchronously,
 *    except for calls that return host data (they synchronise that stream).
 *  - Device-side faults of the method (list overflow, a broken FENE bond, a
 *    non-finite force, a molecule wider than the list allows) are recorded in a
 *    device error word and returned by the next synchronising call (adress_check).
 *  - No call traps, aborts or throws.  Errors are returned as adress_status and
 *    described by adress_last_error.
 */
#ifndef ADRESS_H
#define ADRESS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adress_ctx* adress_handle;

typedef enum {
  ADRESS_OK = 0,
  ADRESS_ERR_ARG = 1,           /* invalid argument or configuration */
  ADRESS_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  ADRESS_ERR_LIST_OVERFLOW = 3, /* more neighbours than the list capacity */
  ADRESS_ERR_NONFINITE = 4,     /* a non-finite force or velocity */
  ADRESS_ERR_BOND_BROKEN = 5,   /* a FENE bond reached its maximum extension */
  ADRESS_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
  ADRESS_ERR_STATE = 7,         /* call out of order (e.g. no state bound) */
  ADRESS_ERR_EXTENT = 8         /* a molecule is wider than the list cutoff allows */
} adress_status;

typedef enum {
  ADRESS_FP64 = 0,      /* every step in double precision */
  ADRESS_FP32_MIXED = 1 /* pair, bonded and thermodynamic forces in float; positions,
                           velocities, energies, virial and density profile in double */
} adress_precision;

/* System description.  Host arrays are copied by adress_init. */
typedef struct {
  int32_t n_mols;        /* M molecules (>= 2) */
  int32_t atoms_per_mol; /* na, 1..4, identical topology for every molecule */
  const double* mass;    /* host [na] per-site masses (> 0) */
  double box[3];         /* periodic box edges L */
  /* resolution function l(d) of d = |x_com - x_center| (minimum image along x):
   * 1 for d < d_at_half, cos^2(pi/2 (d - d_at_half)/d_hy) for d < d_at_half + d_hy,
   * 0 beyond (Sec. "Force interpolation"; squared cosine named in Sec. "Potential
   * energy interpolation") */
  double x_center, d_at_half, d_hy;
  /* atomistic model: WCA between atoms of different molecules,
   * V = 4 eps[(s/r)^12 - (s/r)^6] + eps for r < rc_at */
  double wca_eps, wca_sigma, rc_at;
  /* bonded model (never interpolated): FENE V = -K R0^2/2 ln(1 - r^2/R0^2) on the
   * listed intramolecular pairs, plus WCA on the same pairs when intra_wca != 0 */
  int32_t n_bonds;
  const int32_t* bonds; /* host [2*n_bonds] local atom indices */
  double fene_k, fene_r0;
  int32_t intra_wca;
  /* CG model: COM-COM force F(r) (positive = repulsive) and energy V(r) tabulated on
   * r_k = k*cg_dr, k = 0..cg_n, linear interpolation, zero for r >= rc_cg */
  const double* cg_F; /* host [cg_n+1] */
  const double* cg_V; /* host [cg_n+1] */
  int32_t cg_n;
  double cg_dr, rc_cg;
  /* thermodynamic force F_th(d), nodes d_k = k*tf_dx, linear interpolation; it acts
   * along x (away from the centre when positive) on molecules with
   * d_at_half <= d < d_at_half + d_hy, spread over atoms by mass fraction */
  const double* tf; /* host [tf_n], may be NULL when tf_n == 0 */
  int32_t tf_n;
  double tf_dx;
  /* Langevin thermostat in velocity Verlet: F_L = -gamma m v + sqrt(24 gamma kT m/dt)(u-1/2),
   * u from Philox4x32-10 with key (low, high 32 bits of seed) and counter (atom index within
   * the replica, low and high 32 bits of the time level, 2 replica + block); the FP64 path
   * draws blocks 0 and 1 and forms 53-bit uniforms, the FP32 path takes 24 bits of block 0 */
  double kT, gamma, dt;
  uint64_t seed;
  int64_t replica;
  /* neighbour lists over molecule centres: cutoff max(rc_cg, rc_at + 2 r_ext) + skin between
   * two high-resolution work items, rc_cg + skin when either is coarse-grained */
  double skin, r_ext;
  int32_t max_neighbors; /* initial list capacity per molecule; 0 = automatic */
  int32_t precision;     /* adress_precision */
  /* ---- water-like molecules (all zero: the WCA/FENE model above) ----
   * nb_model 1 (three atoms per molecule): between atoms of different molecules within rc_at,
   * Lennard-Jones with eps_ij = sqrt(lj_eps_i lj_eps_j), sigma_ij = (lj_sigma_i + lj_sigma_j)/2,
   * shifted so that V(rc_at) = 0, plus reaction-field Coulomb
   * V = coulomb_f q_i q_j (1/r + k_rf r^2 - c_rf), k_rf = (eps_rf - 1)/((2 eps_rf + 1) rc_at^3),
   * c_rf = 1/rc_at + k_rf rc_at^2 (wca_eps, wca_sigma unused).  Intramolecular nonbonded
   * pairs are excluded. */
  int32_t nb_model;
  const double* charge;   /* host [na] site charges */
  const double* lj_eps;   /* host [na] >= 0 */
  const double* lj_sigma; /* host [na] */
  double coulomb_f, eps_rf;
  /* bond_model 1: harmonic V = bond_k/2 (r - bond_r0)^2 on the listed pairs (fene_* unused);
   * angles: V = angle_k/2 (theta - angle_theta0)^2 for each (i, vertex j, k), at most 4 */
  int32_t bond_model;
  double bond_k, bond_r0;
  int32_t n_angles;
  const int32_t* angles; /* host [3*n_angles] local atom indices */
  double angle_k, angle_theta0;
  /* ---- self-adjusting geometry (Sec. "Self-adjusting adaptive resolution simulations") ----
   * n_centers > 0 (at most 1024, single-system handles only): the AT region is the union of
   * spheres of radius d_at_half around the resolution centres and the hybrid layer the shells
   * of width d_hy around them; the resolution function takes the distance of the centre of
   * mass to the nearest centre (3D minimum image; the first of equal distances) instead of
   * the slab distance (x_center unused).  The thermodynamic force acts along the direction
   * from that centre; the density profile bins that distance, and the thermodynamic-force
   * update divides the counts by the shell volume around every centre (exact when the
   * spheres do not overlap).  0: the slab. */
  int32_t n_centers;
  const double* centers; /* host [3*n_centers] */
  /* ---- coupling scheme (Sec. "Potential energy interpolation", Eq. Hmix) ----
   * scheme 0: force interpolation (Eq. 1).  scheme 1: energy interpolation (H-AdResS): the
   * pair terms are weighted by (l_a + l_b)/2 instead of l_a l_b, and each hybrid molecule
   * feels the drift force -(V_AT_a - V_CG_a) grad l_a, V_AT_a and V_CG_a being half of its
   * unweighted AT and CG pair energies, spread over its atoms by m_i/M (along x in the slab,
   * along the direction from the nearest centre with resolution centres).  Molecules within
   * r_list of the hybrid layer are then handled as high-resolution work items.  Scheme 1
   * needs the tabulated CG model (no learned CG force).
   * fec_n >= 2 (scheme 1 only): free-energy correction dDF/dl per molecule at fec_n
   * equidistant nodes on l in [0, 1], linear in between; the Hamiltonian gains
   * -sum_a DF(l_a), i.e. the force +g(l_a) grad l_a (not included in the reported
   * energies, like the thermodynamic force).  0: none. */
  int32_t scheme;
  int32_t fec_n;
  const double* fec; /* host [fec_n] */
  /* ---- multiple time stepping (Sec. "Multiple time stepping in adaptive resolution
   * simulations"), impulse r-RESPA ----
   * respa_n > 1 (at most 64): dt is the inner (atomistic) step; the slow forces (CG pair
   * forces, the thermodynamic force and, with energy interpolation, the CG share
   * +(V_CG_a + g(l_a)) grad l_a of the drift force) act as impulses of respa_n dt at every
   * time level divisible by respa_n and not in between.  The force stored in f is
   * F_fast + w F_slow with that weight w; reported energies are unweighted.  0 or 1: off. */
  int32_t respa_n;
} adress_config;

/* Validate `cfg`, copy its tables, allocate the handle's device buffers on the current
 * device and bind `stream` (a cudaStream_t; NULL = legacy default stream).
 * On failure *out is NULL and the status says why. */
adress_status adress_init(const adress_config* cfg, void* stream, adress_handle* out);

/* Batched replicas: n_replicas independent systems in one handle, stepped together by the
 * same kernels (one launch per step over all replicas' molecules, captured in one graph).
 * cfgs[r] describes replica r; the replicas may differ in n_mols, box, x_center,
 * d_at_half, d_hy, replica and the values of tf, and must agree in everything else
 * (ADRESS_ERR_ARG names the first difference).  Replica r's molecules follow those of
 * replicas 0..r-1 in the state arrays (so its atoms are a contiguous range of every
 * component), its lists only hold its own molecules, and each replica's result equals
 * that of a single-system handle with the same config.  The thermodynamic-force table and
 * the density histogram hold tf_n entries per replica, replica after replica; energies and
 * the kinetic observables are sums over all replicas; the rebuild decision is shared (all
 * replicas rebuild when one needs it).  1 <= n_replicas <= 65536, total molecules < 2^23. */
adress_status adress_init_batch(const adress_config* cfgs, int32_t n_replicas, void* stream,
                                adress_handle* out);

/* The state of the method's molecular dynamics (Sec. "Force interpolation": atoms grouped
 * into molecules whose centres of mass carry the resolution).
 * Borrow the caller's device state: x, v double [3][N]; f [3][N] of double
 * (ADRESS_FP64) or float (ADRESS_FP32_MIXED).  Pointers must stay valid until the next
 * bind or adress_destroy.  Rebinding invalidates captured step graphs. */
adress_status adress_bind_state(adress_handle h, double* x, double* v, void* f);

/* Neighbour search of Sec. "Heterogeneous Spatial Domain Decomposition Algorithm" (a
 * linked-cell list over the molecule centres; here on one GPU, with the AT/CG load balance
 * of that section handled by separate work lists instead of non-uniform domains).
 * Map the bound positions to centres of mass and resolution values, then rebuild the
 * Morton-ordered cell list, the class work lists (high-resolution candidates first,
 * then coarse-grained molecules) and the Verlet lists (symmetric; a pair with a
 * coarse-grained item, which has weight 0 until the next build, is listed within
 * rc_cg + skin, a pair of high-resolution items within max(rc_cg, rc_at + 2 r_ext) + skin).
 * Synchronises: grows the list capacity and rebuilds when a molecule has more neighbours
 * than it holds. */
adress_status adress_build_lists(adress_handle h);

/* Conservative forces of the bound positions (Eq. 1 + bonded + thermodynamic force,
 * no thermostat) into f, with a fresh list build.  If energies != NULL (host, 4
 * doubles) synchronises and writes {E_AT, E_CG, E_bond, virial}: E_AT = sum over
 * molecule pairs of w_ab V^AT, E_CG = sum of (1 - w_ab) V^CG with w_ab = l_a l_b (energy
 * interpolation: (l_a + l_b)/2, so that the sum with E_bond is the potential of Eq. Hmix),
 * virial = sum r.f over pair and bond terms.  With multiple time stepping, f carries the
 * slow-force weight of the current time level (see respa_n); the energies do not. */
adress_status adress_compute_forces(adress_handle h, double* energies);

/* Thermostatted dynamics of force interpolation (Sec. "Potential energy interpolation": force
 * interpolation conserves momentum but not energy and needs a thermostat; here Langevin).
 * Advance the bound state (x, v, f at time level n) by nsteps Langevin velocity-Verlet
 * steps:  v += dt/2 f/m;  x += dt v (wrapped);  f = F(x) + F_L(v; n+1);  v += dt/2 f/m.
 * Lists are rebuilt on the device when a molecule centre moved more than skin/2 or a
 * molecule grew wider than the list allows.  Runs as a captured CUDA graph (cached per
 * step count, up to 100 steps per graph): one prologue kernel (half kick, drift,
 * mapping), one fused kernel per further step (forces, thermostat, both half kicks,
 * drift, next mapping), one last kernel (forces, thermostat, second half kick); after each
 * mapping a decide kernel sets the conditional node that runs the list rebuild.  Asynchronous; errors surface at adress_check.
 * With the environment variable ADRESS_EAGER=1 set before adress_init, kernels are
 * launched one by one and the rebuild is decided on the host (synchronising every step);
 * per-kernel profilers cannot see kernels inside graphs that hold conditional nodes. */
adress_status adress_step(adress_handle h, int32_t nsteps);

/* One thermodynamic-force iteration block (Sec. "Free energy corrections and the
 * thermodynamic force": the correction is built from the density profile and refined
 * iteratively): advance nsteps exactly as adress_step does; after every sample_every
 * steps (0 = never) add the folded COM histogram of the positions at that time level to
 * the accumulated profile; at the end, if tf_update != 0, apply one thermodynamic-force
 * iteration with alpha (as adress_tf_update) and reset the profile.  The whole block is
 * one captured CUDA graph (cached per argument set, nsteps <= 1000).  Asynchronous. */
adress_status adress_run(adress_handle h, int32_t nsteps, int32_t sample_every, int32_t tf_update,
                         double alpha);

/* Move the resolution centres of the self-adjusting geometry (n must equal the configured
 * n_centers > 0; host [3n], wrapped into the box): the AT region follows them from the next
 * mapping on, e.g. to track a solute between step calls, and the next step rebuilds the
 * lists.  The resolution of molecules in the hybrid shells changes at once, by up to
 * (pi / (2 d_hy)) times the displacement: move the centres in small increments.
 * Synchronises. */
adress_status adress_set_centers(adress_handle h, const double* centers, int32_t n);

/* Uniform resolution for Kirkwood thermodynamic integration (Sec. "Free energy corrections
 * and the thermodynamic force"): on != 0 gives every molecule l = lambda in [0, 1],
 * independent of its position, so no thermodynamic force, drift force or free-energy
 * correction acts; with energy interpolation H(l) = K + l V_AT + (1 - l) V_CG + V_bond, and
 * the reported E_at and E_cg are l V_AT and (1 - l) V_CG.  on = 0 restores the geometry.
 * The lists must be rebuilt afterwards (adress_build_lists or adress_compute_forces). */
adress_status adress_set_uniform_lambda(adress_handle h, int32_t on, double lambda);

/* Kirkwood thermodynamic integration of energy interpolation (scheme 1, tabulated CG): for
 * each node l_k (host [n], strictly inside (0, 1)): uniform l = l_k, fresh lists and
 * forces, n_equil steps, then n_samples samples every `every` steps of
 * dH/dl = V_AT - V_CG = E_at / l - E_cg / (1 - l); each sample recomputes the conservative
 * force (adress_compute_forces) and the next steps start from it.  dhdl (host [n]) gets the
 * mean per molecule (over all molecules of all replicas), the integrand of
 * DF(l) = int_0^l <V_AT - V_CG>_l' dl' and so a free-energy correction table (fec).  The
 * state advances by n (n_equil + n_samples every) steps; the geometry's resolution, lists
 * and forces are restored at the end. */
adress_status adress_kirkwood(adress_handle h, const double* lambdas, int32_t n, int32_t n_equil,
                              int32_t n_samples, int32_t every, double* dhdl);

/* Radial distribution function numerator of the bound positions: counts (host int64
 * [n_replicas][nbins]) = number of molecule pairs a < b (of the same replica) whose
 * minimum-image centre-of-mass distance r (centres in FP64 as adress_com_lambda computes
 * them) has floor(r / dr) = k < nbins.  All pairs, decided in FP64.  g(r) of bin k is
 * counts_k / (n_samples (M(M-1)/2) (4/3 pi ((k+1)^3 - k^3) dr^3) / V).  The CG model is
 * judged by g(r) (structure) next to forces.  Requires nbins dr <= half of every box edge,
 * nbins <= 4096.  Synchronises. */
adress_status adress_rdf(adress_handle h, int32_t nbins, double dr, int64_t* counts);

/* ---- learned coarse-grained force (force matching) ------------------------------------
 * The CG force of Eq. 1 acts between centres of mass (Sec. "Force interpolation"); the
 * learned variant is a 9 -> 64 -> 64 -> 1 SiLU network of the COM distance d and eight
 * orientation invariants (the projections of each molecule's atoms on the COM axis, each
 * set sorted), trained to reproduce the atomistic force between the two molecules projected
 * on the axis.  It runs on BF16 tensor cores with FP32 accumulation from FP32 master
 * weights; the pair force is the mean over the two orderings of the molecules.
 * params: host float [4865] = W1 [64][9] | b1 [64] | W2 [64][64] | b2 [64] | w3 [64] | b3
 * norm:   host float [19]   = input means [9] | input standard deviations [9] | out_scale
 * force = out_scale * (w3 . silu(W2 silu(W1 (feat - mean)/std + b1) + b2) + b3). */
adress_status adress_mlp_set(adress_handle h, const float* params, const float* norm);
adress_status adress_mlp_get(adress_handle h, float* params, float* norm); /* synchronises */
/* 0: tabulated CG force (default); 1: learned network for every pair with COM distance
 * < rc_cg and l_a l_b < 1 (no CG energy is accumulated in mode 1).  In the MD step the
 * network runs on the tcgen05 tensor cores (128-row products, accumulators in tensor
 * memory); the environment variable ADRESS_MLP_KERNEL=mma, read at the first evaluation,
 * selects the warp-level MMA kernel instead (same results up to summation order). */
adress_status adress_set_cg_mode(adress_handle h, int32_t mode);
/* Append training samples from the bound positions (lists rebuilt first): every molecule
 * pair a < b with COM distance < rc_cg gives features (d, s_a[4], s_b[4]), the atomistic
 * force on a from b along the axis as target, and the ids (a, b); at most cap samples are
 * kept.  *n_total = samples now held.  Synchronises. */
adress_status adress_mlp_collect(adress_handle h, int64_t cap, int64_t* n_total);
/* Copy the first n held samples to the host (any pointer may be NULL). Synchronises. */
adress_status adress_mlp_samples(adress_handle h, float* feat, float* target, int32_t* ids, int64_t n);
/* Replace the held samples by n host samples (features [n][9], targets [n]). Synchronises. */
adress_status adress_mlp_load_samples(adress_handle h, const float* feat, const float* target, int64_t n);
/* Network outputs before out_scale: feat device float [n][9] -> y device float [n]. Async. */
adress_status adress_mlp_forward(adress_handle h, const float* feat, int64_t n, float* y);
/* Mean-squared force-matching loss L = (1/n) sum (y - t/out_scale)^2 of device samples and
 * its gradient: grad host float [4866] = dL/dparams [4865] | n L.  Synchronises. */
adress_status adress_mlp_loss_grad(adress_handle h, const float* feat, const float* target, int64_t n, float* grad);
/* Adam (lr, betas 0.9/0.999, eps 1e-8) over the held samples in mini-batches of `batch`,
 * visiting them in a fixed permutation; loss host float [epochs] = mean loss per epoch.
 * Synchronises. */
adress_status adress_mlp_train(adress_handle h, int32_t epochs, int32_t batch, float lr, float* loss);

/* Force-matched CG table.  The CG force of Eq. 1 acts between the centres of mass
 * (Sec. "Force interpolation"); matched to the atomistic force it is, per COM distance, the
 * mean of the atomistic pair force projected on the COM axis.  From the held samples
 * (adress_mlp_collect: every pair a < b with d < rc_cg, target = that force; or
 * adress_mlp_load_samples):
 *   bins j = floor(d / fit_dr), j < ceil(rc_cg / fit_dr) <= 4096; mean_j = sum of targets /
 *   count over the bins with count >= n_min; F_raw(r) linear between the bin centres
 *   (j + 1/2) fit_dr of those bins, constant below the first and above the last;
 *   F(r_k) = F_raw(r_k) - F_raw(rc_cg) at the table nodes r_k = k cg_dr < rc_cg (so that the
 *   force vanishes continuously at the cutoff), 0 from rc_cg on; V(r_k) = sum over m >= k of
 *   (F_m + F_{m+1}) cg_dr / 2 (trapezoid rule, V = 0 at the last node).
 * F, V: host double [cg_n + 1] (may be NULL).  install != 0 makes it the handle's CG table
 * (both precisions) for the tabulated CG force from the next step on.  Sums are exact
 * (integer accumulation of the targets scaled by 2^48), so the table does not depend on the
 * order of the samples.  Synchronises; ADRESS_ERR_STATE when no samples are held or no bin
 * holds n_min of them. */
adress_status adress_cg_fit(adress_handle h, double fit_dr, int32_t n_min, int32_t install, double* F, double* V);

/* Time level of the bound state (keys the thermostat noise). */
adress_status adress_set_step(adress_handle h, int64_t step);
adress_status adress_get_step(adress_handle h, int64_t* step); /* synchronises */

/* Centres of mass and resolution values of the bound positions: com device double [3][M]
 * (wrapped into the box), w device double [M].  Asynchronous. */
adress_status adress_com_lambda(adress_handle h, double* com, double* w);

/* Kinetic energy and momentum of the bound velocities: out host [4] = {KE, Px, Py, Pz}.
 * Synchronises. */
adress_status adress_kinetic(adress_handle h, double* out);

/* Add the COM histogram of the bound positions, folded about the slab centre, bins of
 * width tf_dx over d = |x_com - x_center| (Sec. "Free energy corrections and the
 * thermodynamic force": the density profile the thermodynamic force is built from).
 * Asynchronous. */
adress_status adress_density_accumulate(adress_handle h);
/* Copy the accumulated counts (host int64 [n], n <= tf_n) and the sample count.
 * Synchronises. */
adress_status adress_density_get(adress_handle h, int64_t* counts, int32_t n, int64_t* nsamples);
adress_status adress_density_reset(adress_handle h);

/* One thermodynamic-force iteration from the accumulated profile, on the device:
 * rho_k = counts_k / (nsamples 2 tf_dx Ly Lz), g_k = (rho_k - rho_{k-1})/tf_dx (g_0 = 0),
 * three-point moving average, tf_k -= alpha * g_k on nodes with
 * d_at_half <= k tf_dx <= d_at_half + d_hy; then resets the histogram.  Asynchronous. */
adress_status adress_tf_update(adress_handle h, double alpha);
adress_status adress_set_tf(adress_handle h, const double* tf_host, int32_t n);
adress_status adress_get_tf(adress_handle h, double* tf_host, int32_t n); /* synchronises */

/* Run-time limits of a handle (which, value):
 *  ADRESS_LIMIT_PAIR_CAPACITY: the learned CG force's pair buffers (set up by
 *    adress_set_cg_mode, sized for every listed pair once: n_mols * capacity / 2) hold at most
 *    min(value, allocation) pairs; value <= 0 restores the allocation.  A step that needs more
 *    pairs evaluates the network for the first `limit` of them only and reports
 *    ADRESS_ERR_LIST_OVERFLOW at the next adress_check; no kernel reads or writes beyond the
 *    buffers.  For memory budgets, and to exercise that error path.
 *  ADRESS_LIMIT_MMA_WAIT_POLLS: polls of the tcgen05 network evaluation's bounded waits for
 *    its tensor-core products (default 2^22, tens of milliseconds); value < 0 restores the
 *    default.  A wait that runs out records ADRESS_ERR_TIMEOUT (reported by adress_check),
 *    the evaluation stops, and each block waits once more with the default limit for the
 *    products it has in flight before it frees its tensor memory; the next evaluation runs
 *    normally.  0 makes every such wait give up at once (for testing the error path).
 * Discards captured graphs.  The paper has no counterpart (resource handling of this
 * implementation). */
typedef enum { ADRESS_LIMIT_PAIR_CAPACITY = 0, ADRESS_LIMIT_MMA_WAIT_POLLS = 1 } adress_limit;
adress_status adress_set_limit(adress_handle h, int32_t which, int64_t value);

/* Copy the current Verlet lists to the host: items host int32 [M] (molecule of each work
 * item, high-resolution candidates first), nn host int32 [M] (neighbour count per item),
 * nbr host int32 [M * capacity] with neighbour slot q of item t at nbr[t * capacity + q].
 * Synchronises.  (Capacity from adress_list_stats.) */
adress_status adress_list_export(adress_handle h, int32_t* items, int32_t* nn, int32_t* nbr);

/* List statistics (host int64 [8]): {n_high_resolution_items, n_cg_items, rebuilds,
 * max_neighbours_at_last_build, capacity, n_cells, 0, 0}.  Synchronises. */
adress_status adress_list_stats(adress_handle h, int64_t* out);

/* Kernel timing for roofline accounting: advances the state by reps + 1 steps with the
 * kernels adress_step uses, launched one by one on the handle's stream with CUDA events
 * around each (prologue, then reps fused steps each followed by a forced list rebuild,
 * then the last step).  ms_out host [4] = milliseconds of {prologue (half kick + drift +
 * mapping), list rebuild (average), fused step (average), last step}.  Synchronises. */
adress_status adress_time_kernels(adress_handle h, int32_t reps, float* ms_out);

/* Launch configuration: threads per block of the mapping and force kernels (32, 64 or
 * 128; 4 threads per molecule) and the list skin (cells have edge >= max(rc_cg, rc_at +
 * 2 r_ext) + skin, so the skin sets the cell size and how often lists are rebuilt).  The
 * results do not depend on either beyond the order of floating-point sums.  Setting them
 * discards captured graphs and the lists (build them again before stepping). */
adress_status adress_set_tuning(adress_handle h, int32_t force_block, double skin);
adress_status adress_get_tuning(adress_handle h, int32_t* force_block, double* skin);

/* Autotuner: for every force_block in {32, 64, 128} and skin in {0.5, 0.75, 1, 1.25, 1.5, 2}
 * x the configured skin (those the boxes admit), run nsteps (1..100) steps of the bound state
 * once to capture the graph and warm up, then 5 times timed with CUDA events; a trial's time
 * is the median of the 5.  The trial with the lowest median is kept if that median is below
 * the fastest of the 5 runs of the setting the call started from; otherwise that setting
 * stays (no change for a gain inside the run-to-run spread).  The bound state (x, v, f, time
 * level) is copied aside first and restored after every trial, and the lists are rebuilt
 * for the chosen pair, so the call leaves the state as it found it.  results (host, may be
 * NULL): up to max_results rows of {force_block, skin, median ms per step, fastest, slowest};
 * *n_results (may be NULL) = rows written.  Synchronises. */
adress_status adress_autotune(adress_handle h, int32_t nsteps, double* results, int32_t max_results,
                              int32_t* n_results);

/* Kinetic energy and momentum of a velocity array without allocating anything: out
 * device double [4] = {KE, Px, Py, Pz} with KE = sum 1/2 m v^2, P = sum m v.
 * The paper has no counterpart; this is a convenience for callers that cannot allocate
 * device memory when they need the observable (a fixed-budget memory pool, an allocator
 * owned by another framework, a monitoring hook that must not change the simulation's
 * allocation pattern): it needs no handle and calls no cudaMalloc, cudaFree or
 * allocating library routine.  Inputs: v device double [3][n_atoms] (the layout of
 * adress_bind_state), atoms_per_mol 1..4 with per-site masses mass (host [atoms_per_mol]),
 * stream (a cudaStream_t, NULL = legacy default stream).  The partial sums live in a
 * file-scope device array of 1024 x 4 doubles (32 KiB) that every GPU loading the library
 * holds until the process exits, which limits n_atoms to 16,777,216 (1024 blocks x 256
 * threads x 64 atoms per thread); larger sizes return ADRESS_ERR_ARG with a message in
 * adress_last_error(NULL).  The first call on a device looks up the array's device
 * address with that device current (cudaGetSymbolAddress); make that first call before
 * any stream capture.  The address is kept for the life of the process, which assumes the
 * device's primary context is never reset (no cudaDeviceReset) while the library is
 * loaded.  All calls share the one array and it keeps the last call's
 * contents: calls that overlap on the GPU (other streams, other host threads) race.
 * Asynchronous on `stream`; errors are returned as adress_status. */
adress_status adress_kinetic_noalloc(const double* v, int64_t n_atoms, int32_t atoms_per_mol,
                                     const double* mass, void* stream, double* out);

/* Synchronise the stream and return (then clear) the first device-side error. */
adress_status adress_check(adress_handle h);

/* Message for the last failing call on h (or for init failures when h == NULL). */
const char* adress_last_error(adress_handle h);
const char* adress_status_string(adress_status s);

/* Free everything the handle owns.  Synchronises its stream first. */
void adress_destroy(adress_handle h);

#ifdef __cplusplus
}
#endif
#endif /* ADRESS_H */
