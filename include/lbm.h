/*
 * liblbm: GPU (sm_103a) reactive lattice Boltzmann step for a carrier gas and
 * reactant/product species on a voxelised porous catalyst.
 *
 * Method: Falcucci et al., "Mapping Reactive Flow Patterns in Monolithic
 * Nanoporous Catalysts" (2016).
 *   - lattice BGK equation for every species with one omega = 1/tau
 *     (Appendix, Eq. LBE); second-order equilibrium (Appendix, Eq. feq) on
 *     the D3Q19 lattice; moments (Appendix, moment equation);
 *   - species transported with the carrier velocity (Sec. 3: the carrier
 *     takes reactant and product along passively), or optionally every
 *     array relaxed towards the barycentric velocity (Appendix, velocity
 *     equation);
 *   - halfway bounce-back of the inert carrier at solid links;
 *   - catalytic "sputtering" boundary condition at every solid node touching
 *     gas (Appendix, Eq. f_P_in) with the uniform sputtering matrix
 *     S_ij = 1/b(x) over the node's b(x) active links;
 *   - reaction probability from the Damkohler number, Da = tau_ch/(delta/v),
 *     tau_ch = 1/p, v = cs (Sec. 2.3 Eq. Da_def; Sec. 3 after Eq. eff; Table 1),
 *     with delta the measured mean pore chord length;
 *   - conversion efficiency eta (Sec. 3, Eq. eff) and product flux profile
 *     Phi_P (Sec. 3, Eq. Phi_P).
 *
 * Conventions shared by every call:
 *   - cell index c = (z * ny + y) * nx + x (x fastest); x and y periodic.
 *   - D3Q19 direction order: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 =
 *     (+1,+1,0),(-1,-1,0),(+1,-1,0),(-1,+1,0),(+1,0,+1),(-1,0,-1),(+1,0,-1),
 *     (-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1); opposite pairs
 *     (1,2),(3,4),...
 *   - species arrays: 0 = carrier C, 1 = reactant R, 2 = product P.
 *   - every function returns 0 (LBM_OK) or a negative LBM_ERR_* code and
 *     never aborts or throws; lbm_error_string() names the code and
 *     lbm_last_error() gives the message of the calling thread's last error.
 *   - handles are owned by the library and freed by their destroy call.
 *   - device memory comes from the caller's lbm_allocator when one is given,
 *     otherwise from cudaMallocAsync on the handle's stream.
 *   - work is enqueued on the handle's stream (a cudaStream_t passed as
 *     void*); only calls that return host data synchronise that stream.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_ARG -1      /* bad argument (null pointer, size, range) */
#define LBM_ERR_OOM -2      /* device allocation failed */
#define LBM_ERR_CUDA -3     /* a CUDA call failed (message in lbm_last_error) */
#define LBM_ERR_DIVERGED -4 /* NaN or non-positive carrier density found */
#define LBM_ERR_STATE -5    /* call not valid in the handle's current state */
#define LBM_ERR_TIMEOUT -6  /* a bounded in-kernel wait ran past its limit */

/* population storage: every format holds the scaled deviation from the rest
 * state, d = (f - w rho_ref) / w with rho_ref = 1 (carrier) or 0 (species),
 * in two arrays: the carrier, and the species (reactant and product of one
 * slot side by side). Collisions run in FP32 on d; FP64 only in the
 * observables' reductions. */
#define LBM_FP32 0     /* d stored as float */
#define LBM_FP16_DEV 1 /* IEEE binary16: the carrier rounded to nearest even;
                          the species, scaled by 2^14, rounded stochastically
                          (unbiased: up with probability equal to the dropped
                          fraction, from reproducible counter-based random
                          bits per entry, slot and step) */
#define LBM_BF16_DEV 2 /* bfloat16: every array rounded stochastically */

/* addressing */
#define LBM_LAYOUT_AUTO 0  /* fluid-only when the fluid fraction is below 0.98 (measured crossover) */
#define LBM_LAYOUT_DENSE 1 /* populations for every cell, solid lanes idle */
#define LBM_LAYOUT_FLUID 2 /* populations for fluid cells only, indirect */

/* z boundary */
#define LBM_BC_PRESSURE 0 /* planes z=0 / z=nz-1 are inlet / outlet planes */
#define LBM_BC_PERIODIC 1 /* z periodic, no inlet or outlet (closed box) */

/* fields for lbm_get_field */
#define LBM_FIELD_RHO_C 0
#define LBM_FIELD_RHO_R 1
#define LBM_FIELD_RHO_P 2
#define LBM_FIELD_UX 3
#define LBM_FIELD_UY 4
#define LBM_FIELD_UZ 5
#define LBM_FIELD_DRHO_C 6 /* rho_C - 1 at full FP32 relative precision */

typedef struct lbm_geometry lbm_geometry;
typedef struct lbm_sim lbm_sim;

/* Caller-provided device allocator (e.g. a framework's caching allocator).
 * alloc returns NULL on failure; both receive the handle's stream. */
typedef struct {
  void *ctx;
  void *(*alloc)(void *ctx, size_t bytes, void *stream);
  void (*free)(void *ctx, void *ptr, size_t bytes, void *stream);
} lbm_allocator;

/* Geometry description (caller-owned; read during lbm_create_geometry only).
 * The synthetic np-Au stand-in: inside the slab z in [slab_z0, slab_z1) the
 * cells with the round-half-even(porosity * slab cells) smallest values of a
 * periodic integer Gaussian random field are fluid (ties: lower index),
 * everything else in the slab is solid, and cells outside the slab are fluid.
 * The field is white noise (sum of 12 uniform 16-bit draws from SplitMix64 of
 * seed ^ (12 c + k), centred) smoothed by 3 periodic box passes per axis of
 * odd width W = nearest odd integer to sqrt(2 corr_len^2 + 1).
 * When mask is non-NULL it is used instead (host array of nx*ny*nz bytes,
 * copied): 0 fluid, 1 catalytic solid, 2 inert solid (never a node: every
 * array bounces back from it halfway, as the carrier does from any solid;
 * the non-reactive plate of the Appendix's validation channel). With LBM_BC_PRESSURE no solid may lie within one cell
 * of the planes z=0 and z=nz-1 (planes 0, 1, nz-2, nz-1 all fluid). */
typedef struct {
  int32_t nx, ny, nz;
  int32_t slab_z0, slab_z1;
  double porosity, corr_len;
  uint64_t seed;
  const uint8_t *mask;
  int32_t bc_z; /* LBM_BC_PRESSURE or LBM_BC_PERIODIC */
  /* Sub-domain of a decomposition along z (0 for a whole box). halo_lo /
   * halo_hi = 1: the two planes at that end (z = 0, 1 / nz-2, nz-1) are a
   * halo copied from the neighbouring sub-domain: never stepped, may hold
   * solid, with no inlet or outlet condition at that end. The inner halo
   * plane (1 / nz-2) exchanges populations and wall hits with the neighbour
   * (lbm_halo_pops, lbm_halo_hits); the outer one (0 / nz-1) only completes
   * the links of the inner plane's catalytic nodes. Needs LBM_BC_PRESSURE
   * and a caller mask. entry_base: the lattice entries of the whole box
   * before this sub-domain's plane 0 (fluid cells with fluid-only
   * addressing, cells with dense), so that the stochastic rounding draws
   * what the whole box would; z_base: the whole box's z of plane 0. */
  int32_t halo_lo, halo_hi;
  int64_t fluid_base;  /* fluid cells of the whole box in planes below z_base */
  int32_t z_base;
} lbm_geometry_desc;

/* Simulation parameters (caller-owned; read during lbm_init only). */
typedef struct {
  double tau;          /* BGK relaxation time of every species (> 0.5) */
  double rho_in;       /* carrier density imposed on the inlet plane */
  double rho_out;      /* carrier density on the outlet plane; initial density */
  double c_in;         /* reactant density imposed on the inlet plane */
  double Da;           /* Damkohler number -> p = min(1, cs / (Da delta)) */
  double p_override;   /* if in [0, 1], used as p instead of the Da mapping */
  double pS_R, pS_P;   /* sticking probabilities (Table 1: 0.95, 0.0) */
  int32_t n_species;   /* 1 = R only, 2 = R and P (besides the carrier) */
  int32_t storage;     /* LBM_FP32 / LBM_FP16_DEV / LBM_BF16_DEV */
  int32_t layout;      /* LBM_LAYOUT_AUTO / _DENSE / _FLUID */
  int32_t deterministic; /* 1: wall hits summed in 64-bit fixed point (2^-58),
                            exact in any order, so a simulation evolves
                            bit-identically alone, in a batched launch or
                            split into sub-domains; 0 (default): FP32 sums
                            in a fixed link order per node (reproducible run
                            to run; a sub-domain's cut nodes add the
                            neighbour's share in another order) */
  int32_t sputter;     /* LBM_S_UNIFORM (default): S_ij = 1/b(x) over the
                          node's active links; LBM_S_RANDOM: the Appendix's
                          random matrix with one-hot columns, each species
                          population reaching a catalytic node re-emitted
                          whole along one active link drawn uniformly per
                          (node, incoming link, step) from sputter_seed
                          (Appendix, Eq. f_P_in and the sentences after it);
                          LBM_S_BOUNCEBACK: no catalysis, the species bounce
                          back at every solid as the carrier does (the
                          non-reactive reference) */
  uint64_t sputter_seed;
  int32_t velocity;    /* velocity u of every array's equilibrium feq(rho_a, u):
                          LBM_U_CARRIER (default): the carrier's own,
                          u = j_C / rho_C, the species carried along
                          passively (Sec. 3); LBM_U_BARYCENTRIC: the mixture's,
                          u = sum_a j_a / sum_a rho_a over carrier and species
                          (Appendix, velocity equation), so that collisions
                          conserve the total momentum. The exported u fields
                          and Phi_P use the same u */
  int32_t inlet;       /* LBM_INLET_PRESSURE (default): the inlet plane z = 0
                          takes feq(rho_in, u) and R feq(c_in, u), u the
                          velocity of plane 1 at the previous step;
                          LBM_INLET_VELOCITY: the same densities at the fixed
                          velocity u = (0, 0, u_in) (Sec. 3: carrier and
                          reactant injected at a constant speed U_in). Needs
                          LBM_BC_PRESSURE geometry (open z) */
  double u_in;         /* inlet speed along +z, |u_in| <= 0.3 (velocity inlet) */
  double tau_s;        /* relaxation time of the reactant and product
                          (diffusivity cs^2 (tau_s - 1/2)); 0 (default): the
                          carrier's tau; else > 0.5 */
  double g_z;          /* body-force acceleration along +z on the carrier
                          (Appendix, validation channel), |g_z| <= 0.01, with
                          the forcing of Guo, Zheng and Shi (2002): the
                          velocity is j/rho + g_z/2 and the collision adds
                          (1 - omega/2) w_i [3 (c_i - u) + 9 (c_i . u) c_i] . F,
                          F = rho g. Needs LBM_U_CARRIER and LBM_FP32
                          storage (the per-step increment is below the
                          16-bit formats' resolution) */
  int32_t desorb;      /* 0 (default): the printed law, stuck unreacted
                          reactant is lost (R re-emitted with 1 - pS_R);
                          1: it desorbs (R re-emitted with 1 - p pS_R), so
                          R + P is conserved when pS_P = 0 */
  double c_init;       /* initial reactant density in every fluid cell, at
                          rest (species equilibrium w_i c_init in each
                          population, except the populations that arrive from
                          catalytic solid, which the walls have not yet
                          re-emitted: 0); 0 (default) is the paper's start
                          with no reactant or product inside the domain
                          (Sec. 3). A positive value starts with the
                          catalytic boundary active everywhere, as after the
                          reactant has filled the pores */
} lbm_params;
#define LBM_S_UNIFORM 0
#define LBM_S_RANDOM 1
#define LBM_S_BOUNCEBACK 2
#define LBM_U_CARRIER 0
#define LBM_U_BARYCENTRIC 1
#define LBM_INLET_PRESSURE 0
#define LBM_INLET_VELOCITY 1

/* Observables (caller-owned). Scalars are FP64 results of device
 * reductions. Profile pointers are optional caller host arrays of nz doubles
 * (NULL = skip); site_map is an optional host array of n_nodes floats. */
typedef struct {
  int64_t step;
  double M_C, M_R, M_P;          /* mass in the interior planes 1..nz-2 (all planes if z periodic) */
  double eta;                    /* sum rho_P(z=nz-2) / sum rho_R(z=1)  (Eq. eff) */
  double in_C, in_R, in_P;       /* cumulative flow through the inlet face into plane 1 */
  double out_C, out_R, out_P;    /* cumulative flow through the outlet face out of plane nz-2 */
  double hits_R, hits_P;         /* cumulative species mass that reached catalytic nodes */
  double reacted;                /* p pS_R hits_R */
  double stuck_R, stuck_P;       /* pS_R (1 - p) hits_R, pS_P hits_P */
  double resid_C, resid_RP;      /* mass-balance residuals (0 up to rounding) */
  double delta, p, Kn;           /* chord length, reaction probability, Knudsen number */
  double *rhoC_z, *rhoR_z, *rhoP_z; /* per-plane density sums */
  double *phiP_z;                   /* per-plane sum rho_P u_z   (Eq. Phi_P) */
  double *react_z;                  /* per-plane p pS_R A^R of the last step */
  float *site_map;                  /* p pS_R A^R per catalytic node, node order */
} lbm_obs;

/* Build a geometry on the device: the voxelised porous catalyst (the
 * paper's nanoporous-gold sample, Sec. 2.1; here the synthetic field above or
 * a caller mask) and the structures the step needs: fluid and catalytic-node
 * numbering, the active links b(x) of each node (Appendix, the normalisation
 * of the sputtering matrix) and the mean pore chord length delta that maps
 * Da to p (Sec. 2.3). stream: cudaStream_t (may be NULL = legacy
 * default stream); alloc: optional. Synchronises the stream. Errors:
 * LBM_ERR_ARG (sizes, slab outside [0,nz], porosity outside [0,1], solid next
 * to an inlet/outlet plane), LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_create_geometry(const lbm_geometry_desc *desc, void *stream, const lbm_allocator *alloc,
                        lbm_geometry **out);

/* Counts: fluid cells, catalytic (interface) nodes, fluid->catalytic links, and
 * the mean pore chord length of the slab, delta = 3 N_fluid / (fluid runs
 * along x, y and z), x and y runs periodic, z runs clipped to the slab. */
int lbm_geometry_info(const lbm_geometry *g, int64_t *n_fluid, int64_t *n_nodes, int64_t *n_links,
                      double *delta);

/* Copy derived integer structures to caller host buffers (NULL = skip):
 * mask[n] (0 fluid, 1 catalytic solid, 2 inert solid); fluid_idx[n] (fluid
 * number in linear order or -1); node_idx[n] (catalytic node number in
 * linear order or -1); b[n] (active links of each catalytic solid cell, 0
 * otherwise); links[n_links][3] = (fluid cell, direction i, catalytic solid
 * cell c + c_i) ordered by cell then i. */
int lbm_geometry_export(const lbm_geometry *g, uint8_t *mask, int32_t *fluid_idx, int32_t *node_idx, int32_t *b,
                        int64_t *links);

void lbm_geometry_free(lbm_geometry *g);

/* Device bytes a simulation of this geometry and these parameters holds. */
int lbm_footprint(const lbm_geometry *g, const lbm_params *prm, size_t *bytes);

/* Upper bound of the device bytes a request needs before its geometry
 * exists: the geometry of the described box plus a simulation with these
 * parameters (every cell counted as a fluid cell and a catalytic node). For
 * admission control. */
int lbm_request_footprint(const lbm_geometry_desc *desc, const lbm_params *prm, size_t *bytes);

/* Create a simulation: carrier at rest with density rho_out, no species
 * (the initial state of Sec. 3), reaction probability p from Da by
 * Sec. 2.3 Eq. Da_def with tau_ch = 1/p and v = cs (p = min(1, cs / (Da
 * delta))), or p_override. The geometry must outlive the simulation.
 * Enqueues on stream and synchronises it once. Errors: LBM_ERR_ARG
 * (parameters out of range, a velocity inlet on a periodic box, a plane too
 * large for fluid-only addressing), LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_init(const lbm_geometry *g, const lbm_params *prm, void *stream, const lbm_allocator *alloc,
             lbm_sim **out);

/* Advance nsteps time steps of the lattice BGK equation (Appendix, Eq. LBE
 * with Eq. feq) for the carrier and every species, with halfway bounce-back
 * of the carrier and the sputtering boundary condition (Appendix,
 * Eq. f_P_in) at catalytic solid links, and the inlet/outlet planes. Per
 * step, on the simulation's stream (asynchronous), four launches:
 *   1. the catalytic nodes write the sputtering law's emission into their
 *      links' species slots;
 *   2. a fused collide-stream launch over the warps away from the
 *      inlet/outlet planes, with the halfway bounce-back at solid links
 *      (on odd steps of fluid-only addressing, two launches: first the
 *      region warps of the all-fluid planes, see lbm_warp_counts, then the
 *      others);
 *   3. one over the other warps;
 *   4. the nodes sum the species that reached them (the wall hits).
 * Errors: LBM_ERR_ARG (nsteps < 0), LBM_ERR_CUDA (a launch failed). */
int lbm_step(lbm_sim *s, int64_t nsteps);

/* Measurement support: one step, exactly as lbm_step, with CUDA events
 * recorded around each of its launches. ms[0], ms[1] and ms[2] (three
 * floats) receive the device time in milliseconds of:
 *   [0] the fast kernel (the warps away from the inlet/outlet and halo
 *       planes: plain warps and, in the same launch, the warps whose cells
 *       touch a solid);
 *   [1] the general kernel (the other warps);
 *   [2] the two catalytic-node kernels together (the sputtering law's
 *       emission before the cell updates, the wall hits after them).
 * entries (optional, NULL = skip) receives the lattice entries that the
 * fast and the general kernel update; entries[0] + entries[1] is every
 * lattice entry (dense addressing counts solid entries, which are skipped).
 * Synchronises the simulation's stream. Errors: LBM_ERR_ARG (null simulation
 * or ms), LBM_ERR_CUDA. */
int lbm_step_timed(lbm_sim *s, float *ms, int64_t *entries);

/* Measurement support: how the simulation's lattice warps (32 entries) are
 * divided among the step's kernels, fixed at lbm_init. counts (four
 * int64) receives:
 *   [0] plain warps of the fast kernel (no cell touches a solid), other
 *       than those of [1];
 *   [1] region warps, plain too: fluid-only addressing numbers their cells
 *       and all the cells' neighbours in the cells' own order, up to one
 *       shift, so that their odd steps (a launch of their own) form the
 *       neighbours' entries by arithmetic instead of reading the fluid
 *       index;
 *   [2] wall warps of the fast kernel (some cell touches a solid);
 *   [3] warps of the general kernel (inlet/outlet and halo planes).
 * Warps with no live entry are not counted. Errors: LBM_ERR_ARG (null
 * simulation or counts). */
int lbm_warp_counts(const lbm_sim *s, int64_t *counts);

/* Advance n simulations by nsteps steps each (continuous batching of small
 * simulations). Simulations of equal storage, layout, species count and
 * accumulation mode form a group of at most 14, whose blocks make up one
 * kernel launch. Simulations at different step parities share a launch.
 * Two launch modes:
 *   LBM_BATCH_PER_STEP (what lbm_step_batch uses): per group and step, the
 *     launches lbm_step makes for one simulation, each over every
 *     simulation of the group: the catalytic nodes' emission, the warps
 *     away from the inlet/outlet planes, the other warps, the nodes' wall
 *     hits;
 *   LBM_BATCH_SINGLE_LAUNCH: one launch per group for up to 1024 steps, one
 *     CTA per (phase, block), three phases per step (emission, cells, wall
 *     hits). Each CTA takes a ticket when it starts; a CTA of a phase waits
 *     until every block of the previous phase has finished. The wait is
 *     bounded (2 s of the GPU's global timer). Measured 1.7-2.4x slower
 *     than per-step launches on GB300: the per-CTA release fences and
 *     acquires of three phases per step cost more than kernel boundaries.
 * The work runs on `stream` (NULL: the first simulation's stream); the caller
 * orders it after any earlier work on the simulations' own streams. Each
 * simulation's result equals what lbm_step would give it alone (bit for bit
 * with deterministic accumulation, else up to the summation order of the
 * wall-hit accumulators), in both modes. Synchronises the stream before
 * returning. Errors: LBM_ERR_ARG (null or repeated simulation, simulations
 * on different devices, a simulation of 2^31 / 14 blocks or more, unknown
 * mode), LBM_ERR_OOM (the single-launch mode's step counters, a few KB taken
 * from the first simulation's allocator on `stream` and counted in its
 * lbm_footprint),
 * LBM_ERR_CUDA, LBM_ERR_TIMEOUT (a wait ran past its limit: the simulations
 * of that call are in an undefined state and should be restored from a
 * checkpoint or destroyed). */
#define LBM_BATCH_PER_STEP 0
#define LBM_BATCH_SINGLE_LAUNCH 1
int lbm_step_batch(lbm_sim *const *sims, int n, int64_t nsteps, void *stream);
int lbm_step_batch_mode(lbm_sim *const *sims, int n, int64_t nsteps, void *stream, int mode);

/* Compute observables at the current step (device FP64 reductions, then a
 * small copy to the host; synchronises the stream): masses, the conversion
 * efficiency eta (Sec. 3, Eq. eff), the product flux profile Phi_P (Sec. 3,
 * Eq. Phi_P), the per-layer and per-node reaction of the sputtering law
 * (Appendix, Eq. f_P_in: the reacted share p pS_R of each node's reactant
 * hits) and the mass budgets. Returns LBM_ERR_DIVERGED (after filling *out)
 * when a density is NaN or the carrier mass is <= 0; LBM_ERR_OOM when the
 * site map's staging buffer cannot be allocated; LBM_ERR_CUDA. */
int lbm_observables(lbm_sim *s, lbm_obs *out);

/* Macroscopic field at the current step, dense [n] floats (0 at solid
 * cells; inlet/outlet planes not meaningful). dst is host memory unless
 * dst_on_device != 0. */
int lbm_get_field(lbm_sim *s, int which, void *dst, int dst_on_device);

/* Populations at the current step as FP32 deviations g = f - w rho_ref
 * (rho_ref = 1 for the carrier, 0 for the species), dense
 * [n_species+1][19][n]: the values a plain two-lattice scheme would hold
 * (0 at solid cells; inlet/outlet planes not meaningful). Host dst unless
 * dst_on_device. */
int lbm_get_populations(lbm_sim *s, float *dst, int dst_on_device);

/* Checkpoint / restore. The state is everything a simulation carries between
 * steps: populations, the wall-hit accumulator ring, the inlet/outlet plane
 * cache, the cumulative face flows and wall hits, the step count and the
 * initial masses, behind a header that names the configuration.
 * lbm_state_size gives the bytes; lbm_get_state copies them to caller host
 * memory (synchronises the stream); lbm_set_state restores them into a
 * simulation of the same solid mask, storage, addressing, species count and
 * accumulation mode (LBM_ERR_ARG if the header does not match; the caller's
 * simulation is then unchanged). The physical parameters (tau, densities,
 * Da, sticking) are not part of the state: a restored state continues under
 * the receiving simulation's parameters, which makes a converged flow a warm
 * start for another Da. With equal parameters a restored simulation continues
 * exactly as the original would (bit-identically with deterministic
 * accumulation). The buffer starts with a header of LBM_STATE_HEADER_BYTES
 * bytes; the population array follows it. */
#define LBM_STATE_HEADER_BYTES 136
int lbm_state_size(const lbm_sim *s, size_t *bytes);
int lbm_get_state(lbm_sim *s, void *dst, size_t n);
int lbm_set_state(lbm_sim *s, const void *src, size_t n);

/* Halo exchange of a sub-domain of a z decomposition (geometry halo_lo /
 * halo_hi). Neighbouring sub-domains share two planes at each cut: my first
 * (last) real plane is the neighbour's inner halo, and mine its last (first)
 * real plane. Each step, in this order:
 *   odd steps only, before the step: lbm_halo_pops(s, side, LBM_HALO_PRE,
 *     LBM_HALO_PACK, buf) on both sides of each cut, hand the buffer to the
 *     neighbour, lbm_halo_pops(..., LBM_HALO_PRE, LBM_HALO_UNPACK, buf) with
 *     the neighbour's;
 *   the step (lbm_step(s, 1));
 *   odd steps only: the same with LBM_HALO_POST;
 *   every step: lbm_halo_hits(s, side, LBM_HALO_PACK, buf), hand it over,
 *     lbm_halo_hits(..., LBM_HALO_UNPACK, buf) (adds the neighbour's wall
 *     hits of the shared planes' catalytic nodes to mine, so both hold the
 *     totals the sputtering law re-emits; in 64-bit fixed point, with
 *     deterministic accumulation, the totals equal the whole box's bit for
 *     bit).
 * A PRE buffer holds the 5 populations per array that cross the cut (c_z
 * towards the neighbour) of the real plane, a POST buffer those of the inner
 * halo plane that this sub-domain's step wrote; POST unpacking skips the
 * slots whose upwind cell is solid. side: LBM_HALO_LO (the neighbour below)
 * or LBM_HALO_HI. buf: device memory of lbm_halo_bytes bytes, in the same
 * order on both sides. All work is enqueued on the simulation's stream.
 * Errors: LBM_ERR_ARG (no halo at that side, random sputtering matrix,
 * null buffer, bad phase or direction), LBM_ERR_CUDA. */
#define LBM_HALO_LO 0
#define LBM_HALO_HI 1
#define LBM_HALO_PRE 0
#define LBM_HALO_POST 1
#define LBM_HALO_PACK 0
#define LBM_HALO_UNPACK 1
int lbm_halo_bytes(const lbm_sim *s, int side, size_t *pop_bytes, size_t *hit_bytes);
int lbm_halo_pops(lbm_sim *s, int side, int phase, int dir, void *buf);
int lbm_halo_hits(lbm_sim *s, int side, int dir, void *buf);

/* Self-test of the bounded wait used by lbm_step_batch: `ctas` CTAs (1..8)
 * each count their arrival, then wait until `expected` (1..64) arrivals are
 * counted. With expected <= ctas every wait ends and the call answers
 * LBM_OK; with expected > ctas no wait can end, every CTA gives up after
 * timeout_s seconds (0 < timeout_s <= 10) and the call answers
 * LBM_ERR_TIMEOUT, with the context intact. *passed receives the number of
 * CTAs whose wait ended. Synchronises the stream. */
int lbm_selftest_barrier(int ctas, int expected, double timeout_s, void *stream, int *passed);

/* Bounds checks of a library built with -DLBM_CHECKED (a debugging aid):
 * *word receives the first out-of-bounds access that any kernel of this
 * process detected since the last call, as kind << 56 | element index
 * (kind 1 populations, 2 wall-hit accumulators, 3 geometry index, 4 plane
 * cache, 5 node tables; 0: none), and the record is cleared. The checked
 * kernels send such an access to element 0 of the same buffer instead.
 * The default build has no checks and returns LBM_ERR_STATE. */
int lbm_check_status(uint64_t *word);

/* Simulation info: step count, storage, layout actually used, p. */
int lbm_sim_info(const lbm_sim *s, int64_t *step, int *storage, int *layout, double *p);

void lbm_destroy(lbm_sim *s);

/* Largest nz that lbm_observables_noalloc accepts. */
#define LBM_NOALLOC_MAX_PLANES 4096

/* lbm_observables for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is a deployment variant. Some callers
 * run the library inside a fixed memory budget, such as a serving loop that
 * admits simulations by their lbm_footprint and must not see an extra
 * allocation when it polls conversion, or an application whose allocator
 * must not be entered from the polling thread. lbm_observables may stage the
 * site map in a temporary device buffer; this call never allocates (no
 * cudaMalloc, no allocator callback, no host heap). Its reduction scratch
 * (per-plane FP64 sums, column totals) is a fixed device array of about
 * 360 KB, sized for LBM_NOALLOC_MAX_PLANES planes, that every GPU loading
 * the library holds until the process exits.
 *
 * Results equal those of lbm_observables (same kernels, same summation
 * order). Arguments as for lbm_observables, except that out->site_map must
 * be NULL. Errors: LBM_ERR_ARG for a null argument, nz above
 * LBM_NOALLOC_MAX_PLANES or a non-NULL site_map; LBM_ERR_CUDA;
 * LBM_ERR_DIVERGED as for lbm_observables. This call does not update
 * lbm_last_error().
 *
 * The first call on a device looks up the scratch array's device address
 * (once per device, with the simulation's device made current for the
 * lookup); make that first call before any stream capture. The address is
 * kept for the life of the process: do not use this call after
 * cudaDeviceReset() (or anything else that destroys the device's primary
 * context), whose new context would hold the array elsewhere. Every call on a
 * device shares the one scratch array: calls that overlap on the GPU (from
 * two streams or two host threads at once) race and must be serialised by
 * the caller. Synchronises the simulation's stream. */
int lbm_observables_noalloc(lbm_sim *s, lbm_obs *out);

const char *lbm_error_string(int code);
const char *lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
