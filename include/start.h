/*
 * start.h -- C ABI of the GB300 (sm_103a) implementation of the START
 * radiative-transfer hot path (Hasegawa & Umemura 2010, "START: Smoothed
 * particle hydrodynamics with tree-based accelerated radiative transfer").
 *
 * The hot path, per time step:
 *   1. frame + Morton keys of particles and sources; stable sort      (Sec. 2.2.2)
 *   2. source octree, one source per leaf by default                  (Sec. 2.2.2)
 *   3. luminosity moments: L = sum L_j, r = sum L_j r_j / sum L_j      (Sec. 2.2.2)
 *   4. particle octree and neighbour lists N(i) = {k : |r_k-r_i| < 2h_i}
 *                                                                     (Sec. 2.2.1)
 *   5. per target: walk the source tree, accepting a cell when
 *      l/d <= theta_crit and its parent was not accepted              (Eqs. con1, con2)
 *   6. per accepted cell / individual source: optical depth by upstream
 *      ray marching, tau_t = tau_up + sigma dl (n_t + n_up)/2          (Eq. tau, Sec. 2.2.1)
 *   7. Gamma_i = sum L e^-tau / (4 pi r^2)                             (Eq. solution2, ksum)
 *   8. implicit hydrogen ionisation update                             (Appendix A)
 *   9. diffuse mode: every particle also emits N_rec = alpha_1 n_e n_p V
 *      and receives the self term k_self                               (Sec. 4.1, Eqs. ssum, kself1)
 *
 * Readings of points the paper leaves open (identical in the library and
 * in its test oracle):
 *   - d in con1 is the Euclidean distance from the target to the cell cube
 *     (0 inside); the root is tested by con1 alone; a leaf that is not
 *     accepted contributes its sources one by one.
 *   - the upstream particle of j toward a source at r_s is the neighbour k
 *     strictly closer to r_s maximising (r_s-r_j).(r_k-r_j)/|r_k-r_j|
 *     (smallest angle), ties to the smaller input index; a chain with no
 *     closer neighbour ends with sigma n_j |r_j - r_s|.
 *   - dl = |r_j - r_s| - |r_up - r_s|; n is the neutral density n_HI.
 *   - r in the dilution is floored at 1e-6 of the root cube side.
 *   - hydrogen only, isothermal; alpha_B on the spot, alpha_A (and the
 *     diffuse emitters) in diffuse mode; one backward-Euler step in the
 *     neutral fraction y = 1 - x_HII per call.
 *
 * Conventions for every function below:
 *   - Return value: START_OK (0) or a negative START_E* status; no
 *     exception crosses the ABI.  start_last_error() describes the last
 *     failure of a context.
 *   - Pointers may address host or device memory (anything the CUDA
 *     runtime can address under unified virtual addressing).  Inputs are
 *     copied into library-owned device buffers; the caller keeps ownership
 *     and may free or reuse them when the call returns.  Outputs in device
 *     memory are written by stream-ordered kernels and are valid once the
 *     context's stream is synchronised; outputs in host memory are valid
 *     when the call returns (the call synchronises the stream).
 *   - All work is issued on start_params.stream (NULL = legacy default
 *     stream) of the current CUDA device at start_create.
 *   - Positions are float32, structure-of-arrays (x[0..n), y[0..n),
 *     z[0..n)) in units of len_unit_cm.  Luminosities are float64 photons
 *     per second (they exceed float32's range).  Gamma is float32 photons
 *     cm^-2 s^-1.  Neutral fractions y are float64.
 *   - Particle arrays are in the caller's (input) order on both sides of
 *     the ABI; the library works internally in Morton order.
 */
#ifndef START_H
#define START_H

#ifdef __cplusplus
extern "C" {
#endif

#define START_OK 0
#define START_EINVAL (-1)     /* invalid argument: NaN/Inf, h <= 0, L < 0, theta < 0, ... */
#define START_ENOMEM (-2)     /* device allocation failed */
#define START_ENOTBUILT (-3)  /* start_build_trees / start_set_state not called yet */
#define START_ECUDA (-4)      /* a CUDA runtime call failed */
#define START_ETIMEOUT (-5)   /* a device wait exceeded spin_cap (reserved) */
#define START_ECHAIN (-6)     /* a ray chain exceeded hop_cap */
#define START_ERANGE (-7)     /* a size exceeds the library's limits (N >= 2^30) */

#define START_DIFFUSE 1u      /* start_build_trees flag: particles also emit */

#define START_MAX_N (1LL << 30)

/* Run parameters.  start_default_params fills the values of the
 * monochromatic 13.6 eV, T = 1e4 K problem with lengths in kpc. */
typedef struct start_params {
    int src_leaf;          /* max sources per source-tree leaf; 1 = the paper's
                              "each cell contains only one radiation source" */
    int ptree_leaf;        /* max particles per particle-tree leaf (neighbour
                              search only; does not change any result) */
    int march_group;       /* lanes cooperating on one neighbour-list
                              evaluation: 1, 2, 4, 8, 16 or 32 (0 = default);
                              does not change any result */
    int timing;            /* 1: record CUDA events around each phase (see
                              start_get_timings); 0: none */
    int march_mode;        /* 1: memoised march, every chain link (virtual
                              source, particle) evaluated once and shared by
                              the rays through it (default); 0: per-ray
                              march, each chain followed from its target.
                              Same upstream choices; tau differs only in the
                              order of the additions */
    int reuse_chains;      /* 1: keep the chain links of a solve resident and,
                              while the particles, sources and theta stay the
                              same, solve later steps from them: only d_tau
                              is recomputed from the current n_HI, the links
                              are summed in chain order, and the step runs as
                              one replayed CUDA graph.  The upstream choices
                              depend on positions only, so the links are
                              those a full solve would find.  Used with the
                              memoised march, without diffuse emitters (whose
                              centres move as x changes) and when the solve
                              fits one target chunk; otherwise ignored */
    double sigma_cm2;      /* HI photoionisation cross-section (6.3e-18) */
    double len_unit_cm;    /* length unit of positions (kpc = 3.0857e21) */
    double L_unit;         /* internal luminosity scale, photons/s (1e48) */
    double alpha_A;        /* case-A recombination coefficient, cm^3/s */
    double alpha_B;        /* case-B recombination coefficient, cm^3/s */
    double tau_cut;        /* per-ray march: rays stop once tau exceeds this
                              (default 110; e^-110 is below float32's smallest
                              subnormal relative to any representable flux) */
    long long hop_cap;     /* max upstream steps per ray (0 = N_p + 1) */
    long long max_pairs;   /* interaction pairs solved at once (bounds the device
                              memory of a solve, about 60 B per pair; 0 = 2^27;
                              a group of a memoised solve holds at most 3.5e9:
                              32-bit link ids).
                              A larger memoised solve is split by virtual source:
                              groups of cells (depth-first index ranges) whose
                              rows are walked and marched over every target at
                              once, so chains are never cut; Gamma's additions
                              are then grouped by them.  The per-ray march splits
                              by Morton-contiguous target chunks instead */
    long long spin_cap;    /* max iterations of any device wait (reserved) */
    void *stream;          /* cudaStream_t to issue work on (NULL = default) */
    double T_eff;          /* 0: monochromatic sources at the Lyman limit (sigma_cm2);
                              else the point sources radiate blackbody spectra of
                              this temperature (K, 500 to 1e7; Test 1 uses 1e5):
                              Gamma becomes sum L F_ion(tau) / (4 pi r^2) and a
                              photoheating rate is kept (start_get_heating) --
                              the photoionisation and photoheating integrals of
                              Appendix A with the hydrogenic cross-section
                              sigma_nu = sigma_cm2 (nu/nu_L)^-3, tau the
                              Lyman-limit depth of the chain.  L stays the
                              ionising photon rate.  Uses the memoised march;
                              reuse_chains is ignored */
    double T_rec;          /* diffuse case: 0 = recombination photons at the
                              Lyman limit; else the (isothermal) gas temperature
                              in K, 100 to 1e5, and the photons of every emitter
                              fill the band nu_L <= nu <= nu_L + k T_rec / h
                              evenly (Section 4.1): emitter rays add
                              L R_ion(tau) / (4 pi r^2) to Gamma, the self term
                              k_self becomes its band average, and the
                              photoheating of the recombination photons (Eqs.
                              gself, gother) joins start_get_heating.  Uses the
                              memoised march */
    int row_warps;         /* tile shape of the memoised march's first hop: target
                              rows per thread block, 4 or 8 (0 = 8); does not
                              change any result */
    int thermal;           /* 0: isothermal, constant alpha_A / alpha_B (above).
                              1: every particle carries a gas temperature
                              (start_set_temperature); start_ionize takes the
                              recombination coefficients at it, adds collisional
                              ionisation, and then advances the temperature by
                              the energy equation of Section 2.1 without its
                              hydrodynamic terms: photoheating from the last
                              solve (start_get_heating) against recombination,
                              free-free, collisional-excitation and collisional-
                              ionisation cooling; the emitters use
                              alpha_1(T) = alpha_A(T) - alpha_B(T).  The rate
                              fits are those of start_ionize's comment */
    int lum_kernel;        /* diffuse case.  0: an emitter cell's luminosity is
                              the sum of its members' (Section 2.2.2, Eq. ssum).
                              1: the kernel-weighted form Section 2.2.2 offers as
                              an alternative, read with the members' emissivity
                              L_j / V_j in place of L_j and the cell's volume as
                              the factor that makes it a luminosity:
                              L = l^3 sum_j (L_j/V_j) W(|r - r_j|, l) / sum_j
                              W(|r - r_j|, l) over the cell's members, r the
                              cell's luminosity centre, W the cubic spline of
                              start_sph_density with h = the cell's edge l; a
                              cell of one member keeps its luminosity */
    int walk_warp;         /* 1: the 32 targets of a warp walk the trees together
                              (one traversal, ballot masks per depth); 0: one
                              independent walk per thread (default: Morton-
                              adjacent targets already walk nearly the same
                              cells, and the shared traversal measured 3 %
                              slower).  Does not change any result */
    int row_bins;          /* upstream search of the memoised march: 0 tests
                              every neighbour of the particle for each link; N
                              in 2..6 (default 4) bins the source direction on a
                              cube map of N x N bins per face and tests only the
                              bin's candidate set -- the neighbours that can
                              still be the upstream choice for some direction in
                              the bin, from bounds on their angle to it (6 N^2
                              64-bit masks per particle, built once per build;
                              lists of at most 64 neighbours).  Links whose
                              source is not farther than every neighbour test
                              them all.  Does not change any result */
    int link_counts;       /* memoised march.  0 (default): the pointer jumping
                              sums each chain's link increments in FP32 over
                              8-byte link states, and start_stats reports hops
                              and max_hops as -1.  1: 16-byte states that also
                              count each chain's links (hops, max_hops) and sum
                              in compensated double-float.  A hop cap
                              (hop_cap > 0) or resident chains (reuse_chains)
                              use the counting form either way */
} start_params;

/* Counters of the last start_rt_solve. */
typedef struct start_stats {
    long long rays;             /* (target, virtual source) pairs evaluated */
    long long hops;             /* chain links over all rays (sum of chain lengths);
                                   -1 when the memoised march did not count them
                                   (start_params.link_counts) */
    long long march_fallbacks;  /* upstream choices decided in FP64 */
    long long walk_fallbacks;   /* opening tests decided in FP64 */
    long long nbr_fallbacks;    /* neighbour tests decided in FP64 (last build) */
    long long nodes_src;        /* nodes of the source tree */
    long long nodes_emit;       /* nodes of the emitter tree (diffuse) */
    long long nodes_part;       /* nodes of the particle tree */
    long long nbr_total;        /* neighbour-list entries */
    long long max_hops;         /* longest chain of the last solve (-1: not counted) */
    long long launches;         /* kernels launched by this context so far */
    long long evals;            /* neighbour-list evaluations performed */
    long long links;            /* distinct chain links (memoised march) */
    long long chunks;           /* target chunks of the last solve */
    long long jump_rounds;      /* pointer-jumping rounds of the last solve (memoised) */
    long long jump_bytes;       /* bytes those rounds read and wrote: s per slot and
                                   round (own state), 2 s per slot that advanced
                                   (first successor read, write), s per further
                                   successor read, s per slot copied once when its
                                   chain closed; s = 8 (16 in the counting form) */
    long long first_hop_scanned;  /* memoised march, every 64th target: candidates
                                     the first hops of its pairs scanned */
    long long first_hop_full;     /* the same targets: neighbours x pairs (what a
                                     scan of every neighbour reads) */
} start_stats;

/* Phases timed when start_params.timing = 1 (milliseconds summed over every
 * occurrence since the previous start_get_timings, from CUDA events on the
 * context's stream; a solve in several target chunks runs the march and
 * Gamma phases once per chunk). */
#define START_PHASE_BUILD 0   /* start_build_trees */
#define START_PHASE_WALK 1    /* interaction lists */
#define START_PHASE_MARCH 2   /* ray march (the dominant kernel) */
#define START_PHASE_GAMMA 3   /* Gamma reduction */
#define START_PHASE_IONIZE 4  /* implicit update */
#define START_PHASE_EMIT 5    /* diffuse emitters and their moments */
#define START_PHASE_HOPS 6    /* memoised march: sum of its hop kernels */
#define START_PHASE_LINK 7    /* memoised march: sum of its link-resolution kernels */
#define START_PHASE_JUMP 8    /* memoised march: sum of its pointer-jumping rounds */
#define START_PHASE_DENSITY 9 /* start_sph_density */
#define START_NPHASES 10

typedef struct start_ctx start_ctx;

/* Fill *p with defaults.  Returns START_EINVAL if p is NULL. */
int start_default_params(start_params *p);

/* Create a context bound to the current CUDA device and p->stream.
 * The library owns the context and every buffer in it. */
int start_create(start_ctx **out, const start_params *p);

/* Release the context and its device buffers (synchronises its stream). */
int start_destroy(start_ctx *c);

/* Replace the parameters of a context (e.g. tuned knobs between requests).
 * The stream and the physical constants may change too; src_leaf and
 * ptree_leaf take effect at the next start_build_trees.  Invalid values give
 * START_EINVAL and leave the context unchanged. */
int start_set_params(start_ctx *c, const start_params *p);

/* Steps 1-4 (and the emitter tree in diffuse mode): frame, keys, sorts,
 * source tree + moments, particle tree, neighbour lists.
 *   pos    [3 * n_p] float32 SoA particle positions
 *   h      [n_p]     float32 smoothing lengths (> 0); neighbours are the
 *                    particles within 2h
 *   src_pos[3 * n_s] float32 SoA source positions
 *   src_L  [n_s]     float64 ionising photons per second (>= 0)
 *   V      [n_p]     float64 particle volumes in len_unit^3 (> 0); required
 *                    with START_DIFFUSE, ignored (may be NULL) otherwise
 *   flags  START_DIFFUSE or 0
 * n_p = 0 or n_s = 0 is allowed.  Sizes >= START_MAX_N give START_ERANGE.
 * Resets the chemistry state to y = 1, n_H = 0 (call start_set_state). */
int start_build_trees(start_ctx *c, const float *pos, const float *h, long long n_p,
                      const float *src_pos, const double *src_L, long long n_s,
                      const double *V, unsigned flags);

/* A batch of independent problems in one context, solved with shared
 * launches: problem b has n_p[b] particles and n_s[b] point sources, its
 * arrays given by pos[b] (SoA 3 x n_p[b]), h[b], src_pos[b], src_L[b] (host or
 * device memory; NULL allowed for empty arrays).  Each problem is built on its
 * own (its frame, source octree and neighbour lists) and the parts are
 * stacked: the context then behaves as one problem of sum n_p particles and
 * sum n_s sources whose particle arrays (n_H, y, n_HI, Gamma, T, ...) are the
 * problems' concatenated in order, and every later call (start_set_state,
 * start_rt_solve, start_ionize, ...) runs one set of kernels over all of
 * them.  A target walks only its own problem's tree and marches only through
 * its own problem's particles, so each problem's results are bitwise those of
 * the same calls on it alone (as long as the batch is not split by max_pairs).
 * Point sources only (no diffuse emitters); resident chains are not kept for
 * a batch; the introspection of the particle tree and of the frame refers to
 * the parts (start_get_frame returns problem 0's).  Costs a context per
 * problem, kept for reuse until start_destroy. */
int start_build_batch(start_ctx *c, int n_problems, const long long *n_p, const long long *n_s,
                      const float *const *pos, const float *const *h,
                      const float *const *src_pos, const double *const *src_L);

/* Resident chemistry state (input order): n_H [n_p] float32 cm^-3 (>= 0),
 * y [n_p] float64 neutral fraction in [0, 1].  Sets n_HI = y n_H. */
int start_set_state(start_ctx *c, const float *n_H, const double *y);

/* Steps 5-7 at opening angle theta (>= 0): Gamma for every particle.
 *   n_HI      [n_p] float32 neutral density (>= 0), or NULL to use the
 *             resident n_HI = y n_H
 *   gamma_out [n_p] float32 photons cm^-2 s^-1, input order; may be NULL
 *             (Gamma is kept resident for start_ionize)
 * In diffuse mode the emitters' luminosities come from the resident state
 * (start_set_state / start_ionize) and the emitter tree adds their
 * photons (self excluded). */
int start_rt_solve(start_ctx *c, const float *n_HI, float theta, float *gamma_out);

/* Step 8: advance the resident y by dt_s seconds with the resident Gamma
 * of the last start_rt_solve (one backward-Euler step), update the
 * resident n_HI, and copy y to y_out [n_p] (input order) when not NULL.
 *
 * With start_params.thermal = 1 (the temperature half of the network of
 * Appendix A, hydrogen only), per particle and in FP64:
 *   1. y: backward Euler of dy/dt = -k y - Gc(T0) n_H y (1 - y)
 *      + alpha(T0) n_H (1 - y)^2 at the step-start temperature T0, k as
 *      above (with alpha_1(T0) in the self term), alpha = alpha_A(T) in the
 *      diffuse case and alpha_B(T) otherwise; the root in [0, 1] of
 *      (a + c) y^2 - (1 + K + c + 2a) y + (y0 + a) = 0 with a = alpha n_H dt,
 *      c = Gc n_H dt, K = k dt;
 *   2. T: backward Euler of the energy density (3/2) (1 + x) n_H k_B T,
 *      (3/2) k_B n_H ((1 + x1) T1 - (1 + x0) T0) = dt (H - Lambda(T1, x1)),
 *      H = y1 n_H h with h the photoheating per neutral atom of the last
 *      solve (0 when every photon is at the Lyman limit), Lambda =
 *      n_e n_p (recombination cooling, case A in the diffuse case, else B,
 *      + free-free) + n_e n_HI (collisional excitation + ionisation
 *      cooling); T1 is kept within [10 K, 1e9 K].
 *   Fits (cgs, lambda = 2 x 157807 K / T): Hui & Gnedin (1997) for
 *   alpha_A, alpha_B, the case A and B recombination cooling and the
 *   collisional ionisation rate Gc (its cooling: k_B 157807 K Gc);
 *   Black (1981) as given by Cen (1992) for collisional excitation
 *   7.5e-19 exp(-118348/T) / (1 + (T/1e5)^0.5); free-free 1.42e-27 g_ff
 *   T^0.5 with g_ff = 1.1 + 0.34 exp(-(5.5 - log10 T)^2 / 3) (Cen 1992). */
int start_ionize(start_ctx *c, double dt_s, double *y_out);

/* Gas temperatures (thermal = 1): T [n_p] float64 kelvin (> 0, finite),
 * input order, host or device.  start_set_state resets every temperature
 * to 1e4 K; start_get_temperature copies the resident ones out. */
int start_set_temperature(start_ctx *c, const double *T);
int start_get_temperature(start_ctx *c, double *T_out);

/* SPH density of Sec. 2.1 (the step before the path when the density
 * changes between solves): rho_i = sum_j m_j W(|r_i - r_j|, h_i) over the
 * particle itself and its neighbours (the particles within 2 h_i of the last
 * start_build_trees, the support of the kernel), with the standard cubic
 * spline W(r, h) = 1/(pi h^3) (1 - 3/2 q^2 + 3/4 q^3) for q = r/h < 1,
 * 1/(pi h^3) (2 - q)^3 / 4 for 1 <= q < 2, 0 beyond.
 *   mass    [n_p] float32 particle masses (>= 0, finite), input order, host
 *           or device; read only
 *   rho_out [n_p] float32, input order, host or device (host: the call
 *           synchronises); mass units per cubed position unit
 * FP32 arithmetic (relative error a few 1e-6).  START_ENOTBUILT before
 * start_build_trees, START_EINVAL for NULL pointers (n_p > 0) or a negative
 * or non-finite mass. */
int start_sph_density(start_ctx *c, const float *mass, float *rho_out);

/* Photoheating rate per neutral hydrogen atom (erg/s), input order, of the
 * last start_rt_solve: sigma_L h nu_L sum L F_heat(tau) / (4 pi r^2) over the
 * point sources with F_heat the spectral integral of the absorbed photons'
 * excess energy h (nu - nu_L) (Appendix A), h nu_L = 13.6 eV.  Point sources
 * at the Lyman limit (T_eff = 0) add nothing: their photons carry no excess
 * energy.  In the diffuse case with the recombination band (T_rec > 0) the
 * recombination photons add
 *   sigma_L h nu_L sum L R_heat(tau) / (4 pi r^2) over the other emitters
 *     (Eq. gother per neutral atom; R_heat the band average of
 *     (nu/nu_L - 1) (nu/nu_L)^-3 e^(-tau (nu/nu_L)^-3)), and
 *   the particle's own absorbed recombination photons (Eq. gself per neutral
 *     atom, from the state of the solve),
 * and nothing when T_rec = 0.  All zero after a solve without spectra.
 * heat_out [n_p] float32, host or device.  START_ENOTBUILT before the first
 * solve. */
int start_get_heating(start_ctx *c, float *heat_out);

/* H2 photodissociation rate of Appendix B for every particle:
 *   k_dis,i = sum over the interaction list of i (point sources only, the
 *             walk of start_rt_solve at theta) of
 *             1.13e8 * F_LW,0 * f_sh(N_H2 / 1e14 cm^-2)  s^-1       (Eq. H2ss)
 *   f_sh(x) = 1 for x <= 1, x^(-3/4) beyond
 *   F_LW,0  = kappa_LW * L / (4 pi r^2): Lyman-Werner photons are not
 *             absorbed by hydrogen atoms, the flux only dilutes
 *   N_H2    = N_H2,up + dl (n_H2,up + n_H2,tar)/2 along the same upstream
 *             chain as tau (Eq. NH2), closed by n_H2 |r_j - r_s| at the
 *             chain end
 *   n_H2     [n_p] float32 cm^-3 (>= 0, finite), input order, host or device
 *   kappa_LW LW specific luminosity per ionising photon per second of a
 *            source (erg s^-1 Hz^-1 per photon s^-1; >= 0): a virtual
 *            source's LW luminosity is kappa_LW times its L
 *   kdis_out [n_p] float32 s^-1, input order, host or device
 * Always uses the memoised march.  The resident Gamma and chemistry state
 * are unchanged; start_get_stats reports this solve.  START_ENOTBUILT before
 * start_build_trees; START_EINVAL for NULL pointers, theta < 0, kappa_LW < 0
 * or a negative or non-finite n_H2. */
int start_h2_dissociation(start_ctx *c, const float *n_H2, float theta, double kappa_LW,
                          float *kdis_out);

/* Stateless form: build + set_state(n_H = n_HI, y = 1) + solve on a
 * temporary context.  Equivalent to the calls above; p may be NULL. */
int start_rt_solve_oneshot(const start_params *p, const float *pos, const float *h,
                           long long n_p, const float *n_HI, const float *src_pos,
                           const double *src_L, long long n_s, float theta,
                           float *gamma_out);

/* ---- introspection (tests, metrics); all outputs may be host memory ---- */

/* Frame: out[0..2] lower corner, out[3] side of the root cube. */
int start_get_frame(start_ctx *c, double out[4]);

/* which = 0 particles, 1 sources.  perm[rank] = input index (sorted order);
 * keys[i] = 63-bit Morton key of input i. */
int start_get_perm(start_ctx *c, int which, unsigned *perm);
int start_get_keys(start_ctx *c, int which, unsigned long long *keys);

/* which = 0 particle tree, 1 source tree, 2 emitter tree.  Nodes are in
 * depth-first pre-order with children in octant order; first/count index
 * the sorted members; skip = index after the node's subtree; cube4 =
 * (lower corner x, y, z, edge) in float64; L = summed luminosity (float64,
 * photons/s); cen3 = luminosity centre in float32.  Any output may be
 * NULL.  start_tree_size returns the node count (or a negative status). */
long long start_tree_size(start_ctx *c, int which);
int start_get_tree(start_ctx *c, int which, int *level, unsigned *first, unsigned *count,
                   unsigned *skip, int *leaf, double *cube4, double *L, float *cen3);

/* Neighbour lists in input order: off [n_p + 1], idx [start_nbr_total]
 * (input indices, any order within a row). */
long long start_nbr_total(start_ctx *c);
int start_get_neighbors(start_ctx *c, unsigned long long *off, unsigned *idx);

/* Interaction lists at theta, rows in input order of the targets:
 * off [n_p + 1]; entries [off[n_p]] may be NULL to query the size.  An
 * entry is the source-tree node id (accepted cell), or
 * START_ENTRY_SOURCE | sorted source rank (member of a leaf that was not
 * accepted); START_ENTRY_EMITTER marks entries of the emitter tree.
 * Entries of one target are in walk order (point sources first). */
#define START_ENTRY_SOURCE 0x80000000u
#define START_ENTRY_EMITTER 0x40000000u
int start_get_lists(start_ctx *c, float theta, unsigned long long *off, unsigned *entries);

/* Checksums of the interaction lists at theta, for comparing them whole at
 * sizes where the lists are too large to copy out: for every target i
 * (input order) hash[i] = 64-bit FNV-1a (offset basis 14695981039346656037,
 * prime 1099511628211) over the entries start_get_lists returns for i, in
 * walk order, each entry fed as its four bytes, least significant first;
 * count[i] = the number of entries.  hash and count are [n_p], host or
 * device memory (count may be NULL).  The walk is the one every solve
 * uses (Eqs. con1, con2). */
int start_get_list_hashes(start_ctx *c, float theta, unsigned long long *hash,
                          unsigned long long *count);

/* Per-particle float32 luminosity of the emitters (input order), photons/s
 * divided by L_unit, as used by the last diffuse solve. */
int start_get_emitter_L(start_ctx *c, float *out);

int start_get_stats(start_ctx *c, start_stats *out);

/* ms[k] = summed duration of phase k (START_PHASE_*) since the previous
 * call, or -1 if it did not run (or timing is off); n entries are written
 * (n <= START_NPHASES).  Resets the sums of every phase.  Synchronises. */
int start_get_timings(start_ctx *c, double *ms, int n);

/* Message of the last failure on c (never NULL). */
const char *start_last_error(const start_ctx *c);

/* Name of a status code. */
const char *start_status_string(int status);

/* Device bytes currently held by all contexts of this process (buffers
 * come from a library-owned stream-ordered pool; a server admits work
 * against a budget with it). */
long long start_memory_in_use(void);

/* The direction bins of start_params.row_bins = N (host only, no device
 * work): a source direction b (nonzero) falls in bin (f N + iu) N + iv,
 * where f = 2 a + (b_a < 0) for the axis a of b's component of largest
 * magnitude, and iu, iv = floor((s / |b_a| + 1) N / 2), clamped to [0, N),
 * for the two other components (s, t) = (b_y, b_z), (b_z, b_x) or (b_x, b_y)
 * on the x, y or z faces.  cones[8 k .. 8 k + 7] receives bin k's cone
 * (unit axis x, y, z, cos rho, sin rho, rho, 0, 0): every direction of the
 * bin lies within rho of the axis (the largest angle to a corner of the
 * bin, widened by 2e-3 rad).  cones holds 48 N^2 floats.  START_EINVAL for
 * N outside 2..6 or a NULL array. */
int start_direction_bins(int N, float *cones);

/* ---- allocation-free Morton ordering (no counterpart in the paper) ----
 *
 * For callers that cannot let the library allocate device memory: codes
 * that hand out all GPU memory from their own pool or a budget fixed at
 * start-up, and codes that must not stall mid-step (cudaMalloc/cudaFree
 * synchronise the whole device).  Computes what start_build_trees computes
 * for a particle set with no sources -- the root frame, the 63-bit Morton
 * key of every particle and the stable order by (key, input index) -- but
 * calls no allocating routine: its scratch is a fixed array compiled into
 * the library, START_NOALLOC_MAX_N particles at most (about 20.5 MB, kept
 * by every GPU that loads this code until the process exits).
 *   pos       [3 * n] float32 SoA positions, device memory
 *   n         0 <= n <= START_NOALLOC_MAX_N (larger: START_ERANGE)
 *   keys_out  [n] Morton keys in input order, device memory
 *   perm_out  [n] input index of each sorted rank, device memory
 *   frame_out [4] lower corner x, y, z and side, device memory or NULL
 *   stream    cudaStream_t to issue the work on (NULL = default stream)
 * Host pointers are refused with START_EINVAL; non-finite positions give
 * START_EINVAL.  The call synchronises `stream` (it reads back the count
 * of non-finite positions) and returns after its work there has finished,
 * so it cannot be issued on a stream that is being captured into a CUDA
 * graph.  The first call on a device also looks up the scratch array's
 * device address (and may load the library's GPU code there).  All calls
 * share the one scratch array, so calls that overlap on the GPU (other
 * streams, other host threads) race; serialise them. */
#define START_NOALLOC_MAX_N (1LL << 20)
int start_morton_order_noalloc(const float *pos, long long n, unsigned long long *keys_out,
                               unsigned *perm_out, double *frame_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* START_H */
