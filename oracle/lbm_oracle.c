/*
 * Plain FP64 CPU oracle for the reactive lattice Boltzmann step.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, includes or
 * calls this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load it. It shares no code, header, table or
 * constant generator with the CUDA path; every table below is written out here
 * on its own.
 *
 * What it computes (Falcucci et al., "Mapping Reactive Flow Patterns in
 * Monolithic Nanoporous Catalysts", 2016):
 *   - lattice BGK equation, one relaxation rate omega = 1/tau for every species
 *     (Appendix, Eq. LBE and the sentence after Eq. feq), or optionally a
 *     rate of their own for the reactant and product
 *     (orc_set_species_tau);
 *   - second-order equilibrium (Appendix, Eq. feq) on the D3Q19 lattice, whose
 *     weights satisfy the constraints of the Appendix (sum w = 1, sum w c = 0,
 *     sum w c c = cs^2 I);
 *   - moments rho = sum f, rho u = sum c f (Appendix, moment equation);
 *   - species advected with the carrier velocity (Sec. 3, initial-condition
 *     paragraph: the carrier takes them along passively), or, optionally,
 *     every array (carrier included) relaxed towards the common barycentric
 *     velocity u = sum_a rho_a u_a / sum_a rho_a of the Appendix's velocity
 *     equation (orc_set_barycentric);
 *   - the catalytic "sputtering" boundary condition (Appendix, Eq. f_P_in) with
 *     the uniform sputtering matrix S_ij = 1/b(x) over the b(x) active links
 *     (its column sums are 1, as the Appendix requires), or, optionally, the
 *     random matrix the Appendix describes, read as one-hot columns: every
 *     species population that reaches a catalytic node is re-emitted whole
 *     along one of the node's active links, drawn uniformly and afresh for
 *     each node, incoming link and step (orc_set_random_sputtering);
 *   - Da -> p through Da = tau_ch / (delta / v), tau_ch = 1/p, v = cs
 *     (Sec. 2.3 Eq. Da_def, Sec. 3 discussion of Eq. eff, Table 1);
 *   - conversion efficiency eta = M_P(outlet plane) / M_R(inlet plane)
 *     (Sec. 3, Eq. eff) and product flux Phi_P = sum rho_P u (Sec. 3, Eq. Phi_P).
 *
 * Streaming is the textbook two-lattice pull form: every fluid cell first
 * collides (f -> fs), every catalytic solid node then gathers the species
 * populations that hit it in this step, and every fluid cell then pulls its
 * new populations from its upwind neighbour, from its own reversed population
 * (carrier, halfway bounce-back) or from the solid node's re-emission
 * (species, sputtering law). Plain loops, no blocking or fusion.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - 3D D3Q19 instead of the paper's 2D D2Q9;
 *   - the carrier (inert, not reactive) bounces back halfway at solid links;
 *   - inlet plane z=0 and outlet plane z=nz-1 are equilibrium planes: the
 *     carrier takes feq(rho_in or rho_out, u) with u the velocity of the
 *     adjacent interior plane at the previous step; species take feq(c_in, u)
 *     at the inlet (product 0) and feq(rho of the adjacent plane, u) at the
 *     outlet; x and y are periodic. Optionally the inlet takes the fixed
 *     velocity (0, 0, u_in) instead (orc_set_velocity_inlet);
 *   - re-emitted species reach the fluid one step after they hit the wall,
 *     with the same timing as bounce-back;
 *   - mask value 2 marks inert solid: not a catalytic node, every array
 *     bounces back from it as the carrier does (the non-reactive plate of
 *     the Appendix's validation channel); optionally every solid is inert
 *     for the species (orc_set_species_bounceback, the non-reactive
 *     reference);
 *   - optionally the stuck, unreacted reactant desorbs instead of being lost:
 *     the reactant is re-emitted with (1 - p pS_R) instead of (1 - pS_R)
 *     (orc_set_desorbing; the variant the Appendix's remark on R + P
 *     non-conservation suggests);
 *   - optional body force on the carrier, acceleration (0, 0, g)
 *     (Appendix, validation: a body force drives the channel flow), by the
 *     forcing scheme of Guo, Zheng and Shi (2002): the velocity is
 *     u = j/rho + g/2 (for every array's equilibrium and for the output), and
 *     the carrier's collision adds (1 - omega/2) w_i [3 (c_i - u) + 9 (c_i . u)
 *     c_i] . F with F = rho g (orc_set_body_force; carrier velocity only).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* D3Q19 lattice: rest, 6 axis links, 12 edge links; opposite pairs (1,2),  */
/* (3,4), ... Weights 1/3, 1/18, 1/36, cs^2 = 1/3.                          */
/* ---------------------------------------------------------------------- */
#define Q 19
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double WQ[Q] = {1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static int opp_of(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
static const double CS2 = 1.0 / 3.0;

void orc_lattice(int *cx, int *cy, int *cz, double *w, int *opp) {
  for (int i = 0; i < Q; ++i) {
    cx[i] = CX[i];
    cy[i] = CY[i];
    cz[i] = CZ[i];
    w[i] = WQ[i];
    opp[i] = opp_of(i);
  }
}

/* Equilibrium of the Appendix (Eq. feq), second order in u. */
static double feq(int i, double rho, double ux, double uy, double uz) {
  double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
  double uu = ux * ux + uy * uy + uz * uz;
  return WQ[i] * rho * (1.0 + cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

void orc_feq(double rho, double ux, double uy, double uz, double *out) {
  for (int i = 0; i < Q; ++i) out[i] = feq(i, rho, ux, uy, uz);
}

/* ---------------------------------------------------------------------- */
/* Reduced-precision storage emulation: round-to-nearest-even to IEEE       */
/* binary16 or to bfloat16, written from the formats' definitions.          */
/* ---------------------------------------------------------------------- */
/* Round x to a multiple of 2^e, ties to even. */
static double round_to_quantum(double x, int e) {
  double scaled = ldexp(x, -e);
  double r = nearbyint(scaled); /* default rounding mode: ties to even */
  return ldexp(r, e);
}

/* binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits; emin = -14,
 * subnormal quantum 2^-24, largest finite 65504. */
double orc_round_fp16(double x) {
  if (x == 0.0 || isnan(x) || isinf(x)) return x;
  double a = fabs(x);
  int e;
  frexp(a, &e); /* a = m 2^e, m in [0.5, 1) -> unbiased exponent e-1 */
  int ue = e - 1;
  if (ue < -14) ue = -14;
  double r = round_to_quantum(x, ue - 10);
  if (fabs(r) >= 65520.0) return copysign(INFINITY, x);
  return r;
}

/* bfloat16: 1 sign, 8 exponent (bias 127), 7 fraction bits. */
double orc_round_bf16(double x) {
  if (x == 0.0 || isnan(x) || isinf(x)) return x;
  double a = fabs(x);
  int e;
  frexp(a, &e);
  int ue = e - 1;
  if (ue < -126) ue = -126;
  return round_to_quantum(x, ue - 7);
}

/* ---------------------------------------------------------------------- */
/* Synthetic np-Au geometry: thresholded integer Gaussian random field.     */
/* ---------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea, Flood 2014): the first output of a generator
 * whose state is x, i.e. mix(x + golden gamma). */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Irwin-Hall white noise: sum of 12 uniform 16-bit integers, centred. */
int64_t orc_noise(uint64_t seed, uint64_t v) {
  int64_t s = 0;
  for (uint64_t k = 0; k < 12; ++k) s += (int64_t)(orc_splitmix64(seed ^ (v * 12 + k)) >> 48);
  return s - 12 * 32768;
}

/* Odd box width W whose 3-pass box filter has the variance of a Gaussian of
 * standard deviation l/sqrt(2): W = nearest odd integer to sqrt(2 l^2 + 1). */
int orc_box_width(double corr_len) {
  double t = sqrt(2.0 * corr_len * corr_len + 1.0);
  int lo = (int)floor(t);
  if (lo % 2 == 0) lo -= 1; /* largest odd <= t */
  if (lo < 1) lo = 1;
  int hi = lo + 2;
  return (t - lo <= hi - t) ? lo : hi;
}

/* One periodic centred box-filter pass of odd width W along axis `ax`,
 * written as the plain sum over the W taps. */
static void box_pass(const int64_t *in, int64_t *out, int nx, int ny, int nz, int ax, int W) {
  int r = W / 2;
  int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
    int64_t s = 0;
    for (int d = -r; d <= r; ++d) {
      int xx = x, yy = y, zz = z;
      if (ax == 0) xx = (int)(((x + d) % nx + nx) % nx);
      if (ax == 1) yy = (int)(((y + d) % ny + ny) % ny);
      if (ax == 2) zz = (int)(((z + d) % nz + nz) % nz);
      s += in[((int64_t)zz * ny + yy) * nx + xx];
    }
    out[c] = s;
  }
}

/* Smoothed field value at every cell: white noise, then 3 box passes per axis. */
void orc_field(int nx, int ny, int nz, double corr_len, uint64_t seed, int64_t *field) {
  int64_t n = (int64_t)nx * ny * nz;
  int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * n);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; ++c) field[c] = orc_noise(seed, (uint64_t)c);
  int W = orc_box_width(corr_len);
  for (int ax = 0; ax < 3; ++ax) {
    for (int pass = 0; pass < 3; ++pass) {
      box_pass(field, tmp, nx, ny, nz, ax, W);
      memcpy(field, tmp, sizeof(int64_t) * n);
    }
  }
  free(tmp);
}

typedef struct {
  int64_t v;
  int64_t idx;
} keyed;

static int cmp_keyed(const void *a, const void *b) {
  const keyed *p = (const keyed *)a, *q = (const keyed *)b;
  if (p->v != q->v) return p->v < q->v ? -1 : 1;
  if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
  return 0;
}

/* Number of fluid cells in a slab of n cells: round-half-even(phi n). */
int64_t orc_fluid_count(double porosity, int64_t n_slab) {
  return (int64_t)llrint(porosity * (double)n_slab);
}

/* Mask (1 = solid): fluid outside the slab z in [z0, z1); inside it the K
 * smallest field values are fluid (ties to the lower linear index). */
void orc_geometry(int nx, int ny, int nz, int z0, int z1, double porosity, double corr_len, uint64_t seed,
                  uint8_t *mask) {
  int64_t n = (int64_t)nx * ny * nz;
  int64_t *field = (int64_t *)malloc(sizeof(int64_t) * n);
  orc_field(nx, ny, nz, corr_len, seed, field);
  int64_t plane = (int64_t)nx * ny;
  int64_t n_slab = plane * (z1 - z0);
  keyed *k = (keyed *)malloc(sizeof(keyed) * (n_slab > 0 ? n_slab : 1));
  for (int64_t c = 0; c < n_slab; ++c) {
    int64_t idx = (int64_t)z0 * plane + c;
    k[c].v = field[idx];
    k[c].idx = idx;
  }
  qsort(k, (size_t)n_slab, sizeof(keyed), cmp_keyed);
  int64_t K = orc_fluid_count(porosity, n_slab);
  memset(mask, 0, (size_t)n);
  for (int64_t c = 0; c < n_slab; ++c) mask[k[c].idx] = (c < K) ? 0 : 1;
  free(k);
  free(field);
}

/* ---------------------------------------------------------------------- */
/* Derived integer structures.                                             */
/* ---------------------------------------------------------------------- */
/* Neighbour of cell (x,y,z) along c_i; x,y periodic; z periodic if zper,
 * else -1 outside [0, nz). */
static int64_t nbr(int nx, int ny, int nz, int zper, int x, int y, int z, int i, int sgn) {
  int xx = ((x + sgn * CX[i]) % nx + nx) % nx;
  int yy = ((y + sgn * CY[i]) % ny + ny) % ny;
  int zz = z + sgn * CZ[i];
  if (zz < 0 || zz >= nz) {
    if (!zper) return -1;
    zz = (zz % nz + nz) % nz;
  }
  return ((int64_t)zz * ny + yy) * nx + xx;
}

/* b(s): number of directions j != 0 with s - c_j a fluid cell (Appendix: the
 * node's active links) for a catalytic solid s (mask 1); 0 for fluid and
 * inert solid cells. */
void orc_active_links(int nx, int ny, int nz, int zper, const uint8_t *mask, int32_t *b) {
  int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
    int cnt = 0;
    if (mask[c] == 1) {
      for (int j = 1; j < Q; ++j) {
        int64_t s = nbr(nx, ny, nz, zper, x, y, z, j, -1);
        if (s >= 0 && !mask[s]) ++cnt;
      }
    }
    b[c] = cnt;
  }
}

/* Fluid index map (fluid cells numbered in linear order, -1 for solid) and
 * interface-node map (solid cells with b >= 1 numbered in linear order, -1
 * otherwise). Returns the counts. */
void orc_index_maps(int nx, int ny, int nz, int zper, const uint8_t *mask, int64_t *fluid_idx, int64_t *node_idx,
                    int64_t *n_fluid, int64_t *n_nodes) {
  int64_t n = (int64_t)nx * ny * nz;
  int32_t *b = (int32_t *)malloc(sizeof(int32_t) * n);
  orc_active_links(nx, ny, nz, zper, mask, b);
  int64_t nf = 0, ns = 0;
  for (int64_t c = 0; c < n; ++c) {
    fluid_idx[c] = mask[c] ? -1 : nf++;
    node_idx[c] = (mask[c] && b[c] > 0) ? ns++ : -1;
  }
  *n_fluid = nf;
  *n_nodes = ns;
  free(b);
}

/* Link list in canonical order: every (fluid cell, direction i) whose target
 * cell + c_i is catalytic solid (mask 1), ordered by cell then direction.
 * Each entry is (fluid linear index, i, linear index of the solid target). Returns the count;
 * writes only if out != NULL. */
int64_t orc_links(int nx, int ny, int nz, int zper, const uint8_t *mask, int64_t *out) {
  int64_t n = (int64_t)nx * ny * nz, m = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (mask[c]) continue;
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
    for (int i = 1; i < Q; ++i) {
      int64_t t = nbr(nx, ny, nz, zper, x, y, z, i, +1);
      if (t >= 0 && mask[t] == 1) {
        if (out) {
          out[3 * m + 0] = c;
          out[3 * m + 1] = i;
          out[3 * m + 2] = t;
        }
        ++m;
      }
    }
  }
  return m;
}

/* Mean pore chord length in the slab: (total fluid length along the three
 * axes) / (number of fluid runs along the three axes) = 3 N_f / R. A run
 * starts at a fluid cell whose predecessor along the axis is solid (x, y
 * periodic; along z, a predecessor outside the slab also starts a run); a
 * periodic line that is fluid everywhere counts as one run. Returns 0 if the
 * slab holds no fluid. */
double orc_chord_length(int nx, int ny, int nz, int z0, int z1, const uint8_t *mask) {
  int64_t nf = 0, runs = 0;
  for (int z = z0; z < z1; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t c = ((int64_t)z * ny + y) * nx + x;
        if (mask[c]) continue;
        ++nf;
        int px = (x + nx - 1) % nx, py = (y + ny - 1) % ny;
        if (mask[((int64_t)z * ny + y) * nx + px]) ++runs;
        if (mask[((int64_t)z * ny + py) * nx + x]) ++runs;
        if (z == z0 || mask[((int64_t)(z - 1) * ny + y) * nx + x]) ++runs;
      }
  /* periodic lines with no solid cell at all */
  for (int z = z0; z < z1; ++z) {
    for (int y = 0; y < ny; ++y) {
      int all = 1;
      for (int x = 0; x < nx; ++x) all &= !mask[((int64_t)z * ny + y) * nx + x];
      runs += all;
    }
    for (int x = 0; x < nx; ++x) {
      int all = 1;
      for (int y = 0; y < ny; ++y) all &= !mask[((int64_t)z * ny + y) * nx + x];
      runs += all;
    }
  }
  if (nf == 0 || runs == 0) return 0.0;
  return 3.0 * (double)nf / (double)runs;
}

/* Da -> p: Da = tau_ch / (delta / cs) with tau_ch = 1/p, so p = cs / (Da
 * delta), clamped to [0, 1] (Da -> 0 is the transport-limited end). */
double orc_reaction_probability(double Da, double delta) {
  double cs = sqrt(CS2);
  if (!(Da > 0.0) || !(delta > 0.0)) return 1.0;
  double p = cs / (Da * delta);
  return p > 1.0 ? 1.0 : p;
}

/* Knudsen number Kn = cs (tau - 1/2) / delta (Sec. 2.3, Eq. knudsen). */
double orc_knudsen(double tau, double delta) { return sqrt(CS2) * (tau - 0.5) / delta; }

/* ---------------------------------------------------------------------- */
/* Simulation state.                                                        */
/* ---------------------------------------------------------------------- */
enum { ORC_BC_PRESSURE = 0, ORC_BC_PERIODIC = 1 };
enum { ORC_Q_NONE = 0, ORC_Q_FP16 = 1, ORC_Q_BF16 = 2 };

typedef struct {
  int nx, ny, nz, zper, ns; /* ns = number of species arrays incl. carrier */
  int64_t n;
  uint8_t *mask;
  int32_t *b;
  double tau, omega, rho_in, rho_out, c_in, p, pSR, pSP;
  double omega_s; /* relaxation rate of the reactant and product */
  double gz;      /* body-force acceleration along z (carrier) */
  int quant;
  double *f;  /* [ns][Q][n] natural populations at time t */
  double *fs; /* [ns][Q][n] post-collision */
  double *A;  /* [2][n] species gathered at solid nodes during the last step */
  int bary;         /* 1: common barycentric velocity of all arrays */
  int vel_in;       /* 1: the inlet plane takes the fixed velocity (0, 0, u_in) */
  int sp_bb;        /* 1: species bounce back at every solid (no catalysis) */
  int desorb;       /* 1: stuck unreacted reactant desorbs */
  double u_in;
  int rs;           /* 1: random (one-hot) sputtering matrix */
  uint64_t rs_seed; /* its seed */
  double *B;        /* [2][Q][n] random sputtering: gathered species by outgoing link */
  double *ubuf_prev, *ubuf_next; /* [2 planes][nx*ny][3 + ns-1]: u, species rho */
  int64_t step;
  /* cumulative, per species: inflow through the inlet face, outflow through
   * the outlet face; sums of A over all steps */
  double F_in[3], F_out[3], A_cum[2];
  double M0[3];
} orc_sim;

static int64_t cidx(const orc_sim *s, int x, int y, int z) { return ((int64_t)z * s->ny + y) * s->nx + x; }

static int is_bc(const orc_sim *s, int z) { return !s->zper && (z == 0 || z == s->nz - 1); }

/* Value a stored population takes in reduced-precision storage: the
 * deviation (f - w rho_ref)/w, rho_ref = 1 for the carrier and 0 for the
 * species, rounded to the storage format. */
static double storeq(const orc_sim *s, int a, int i, double v) {
  if (s->quant == ORC_Q_NONE) return v;
  double ref = (a == 0) ? 1.0 : 0.0;
  double d = (v - WQ[i] * ref) / WQ[i];
  d = (s->quant == ORC_Q_FP16) ? orc_round_fp16(d) : orc_round_bf16(d);
  return WQ[i] * (ref + d);
}

#define F(s, arr, a, i, c) ((arr)[(((int64_t)(a) * Q + (i)) * (s)->n) + (c)])
#define UB_W(s) (3 + (s)->ns - 1)

static void interior_masses(const orc_sim *s, double *M) {
  M[0] = M[1] = M[2] = 0.0;
  for (int a = 0; a < s->ns; ++a) {
    double m = 0.0;
    for (int64_t c = 0; c < s->n; ++c) {
      int z = (int)(c / ((int64_t)s->nx * s->ny));
      if (s->mask[c] || is_bc(s, z)) continue;
      for (int i = 0; i < Q; ++i) m += F(s, s->f, a, i, c);
    }
    M[a] = m;
  }
}

orc_sim *orc_create(int nx, int ny, int nz, int bc_mode, const uint8_t *mask, int n_species, double tau,
                    double rho_in, double rho_out, double c_in, double p, double pSR, double pSP, int quant) {
  orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
  s->nx = nx;
  s->ny = ny;
  s->nz = nz;
  s->zper = (bc_mode == ORC_BC_PERIODIC);
  s->ns = 1 + n_species;
  s->n = (int64_t)nx * ny * nz;
  s->mask = (uint8_t *)malloc((size_t)s->n);
  memcpy(s->mask, mask, (size_t)s->n);
  s->b = (int32_t *)malloc(sizeof(int32_t) * s->n);
  orc_active_links(nx, ny, nz, s->zper, s->mask, s->b);
  s->tau = tau;
  s->omega = 1.0 / tau;
  s->omega_s = s->omega;
  s->rho_in = rho_in;
  s->rho_out = rho_out;
  s->c_in = c_in;
  s->p = p;
  s->pSR = pSR;
  s->pSP = pSP;
  s->quant = quant;
  size_t nf = (size_t)s->ns * Q * s->n;
  s->f = (double *)calloc(nf, sizeof(double));
  s->fs = (double *)calloc(nf, sizeof(double));
  s->A = (double *)calloc((size_t)2 * s->n, sizeof(double));
  size_t nub = (size_t)2 * nx * ny * UB_W(s);
  s->ubuf_prev = (double *)calloc(nub, sizeof(double));
  s->ubuf_next = (double *)calloc(nub, sizeof(double));
  /* initial state: carrier at rest with density rho_out, no species */
  for (int64_t c = 0; c < s->n; ++c) {
    if (s->mask[c]) continue;
    for (int i = 0; i < Q; ++i) F(s, s->f, 0, i, c) = storeq(s, 0, i, feq(i, rho_out, 0, 0, 0));
  }
  interior_masses(s, s->M0);
  return s;
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  free(s->mask);
  free(s->b);
  free(s->f);
  free(s->fs);
  free(s->A);
  free(s->B);
  free(s->ubuf_prev);
  free(s->ubuf_next);
  free(s);
}

/* Set the natural populations of species array a (0 carrier, 1 R, 2 P) at
 * every cell from src[Q][n] (tests use this to prepare worked examples). */
void orc_set_populations(orc_sim *s, int a, const double *src) {
  memcpy(&s->f[(int64_t)a * Q * s->n], src, sizeof(double) * Q * s->n);
  interior_masses(s, s->M0);
}

void orc_get_populations(const orc_sim *s, double *dst) {
  memcpy(dst, s->f, sizeof(double) * (size_t)s->ns * Q * s->n);
}

/* Random sputtering matrix. The Appendix's S_ij is random with unit column
 * sums; the reading taken is a one-hot column per (node, incoming link,
 * step): the population reaching catalytic node `cell` along c_j at step t
 * leaves whole along active link k of the node, where k is drawn uniformly
 * from the node's active links (directions i with cell + c_i fluid) by the
 * SplitMix64 hash (Steele, Lea and Flood 2014) of SplitMix64(seed) xor
 * (t 2^40 + cell 2^5 + j): with h the hash's high 32 bits and b the number
 * of active links, k is the r-th active direction in increasing order,
 * r = floor(h b / 2^32). (Hashing the seed first keeps nearby seeds from
 * sharing keys.) Its mean over draws is the uniform S_ij = 1/b. Returns 0
 * when the node has no active link. */
int orc_rs_choice(uint64_t seed, int64_t cell, int j, int64_t t, uint32_t amask) {
  int b = 0;
  for (int i = 1; i < Q; ++i) b += (amask >> i) & 1u;
  if (b == 0) return 0;
  uint64_t key = ((uint64_t)t << 40) + ((uint64_t)cell << 5) + (uint64_t)j;
  uint64_t h = orc_splitmix64(orc_splitmix64(seed) ^ key) >> 32;
  uint32_t r = (uint32_t)((h * (uint64_t)b) >> 32);
  for (int i = 1; i < Q; ++i)
    if ((amask >> i) & 1u) {
      if (r == 0) return i;
      --r;
    }
  return 0;
}

/* Bit i set: cell + c_i is a fluid cell (the node's active outgoing links). */
static uint32_t out_mask(const orc_sim *s, int64_t c) {
  int x = (int)(c % s->nx), y = (int)((c / s->nx) % s->ny), z = (int)(c / ((int64_t)s->nx * s->ny));
  uint32_t m = 0;
  for (int i = 1; i < Q; ++i) {
    int64_t d = nbr(s->nx, s->ny, s->nz, s->zper, x, y, z, i, +1);
    if (d >= 0 && !s->mask[d]) m |= 1u << i;
  }
  return m;
}

/* Relax every array towards feq(rho_a, u) with u the barycentric velocity
 * sum_a j_a / sum_a rho_a over all arrays, carrier included (Appendix,
 * velocity equation), instead of the carrier's own velocity. */
void orc_set_barycentric(orc_sim *s) { s->bary = 1; }

/* Reactant and product relax with omega_s = 1/tau_s instead of the
 * carrier's 1/tau (diffusivity cs^2 (tau_s - 1/2)). */
void orc_set_species_tau(orc_sim *s, double tau_s) { s->omega_s = 1.0 / tau_s; }

/* Species bounce back at every solid cell, as the carrier does: no node
 * gathers anything and nothing reacts. */
void orc_set_species_bounceback(orc_sim *s) { s->sp_bb = 1; }

/* The stuck, unreacted reactant desorbs: a reactant hit is re-emitted with
 * (1 - p pS_R) as R and p pS_R as P, so R + P is conserved when pS_P = 0. */
void orc_set_desorbing(orc_sim *s) { s->desorb = 1; }

/* Body-force acceleration g along z on the carrier (see the header). */
void orc_set_body_force(orc_sim *s, double gz) { s->gz = gz; }

/* Velocity inlet: the inlet plane's equilibria take the fixed velocity
 * (0, 0, u_in) instead of the velocity of plane 1 at the previous step
 * (Sec. 3: carrier and reactant injected at a constant speed U_in with
 * fixed densities). */
void orc_set_velocity_inlet(orc_sim *s, double u_in) {
  s->vel_in = 1;
  s->u_in = u_in;
}

/* Switch a simulation to the random sputtering matrix (see orc_rs_choice). */
void orc_set_random_sputtering(orc_sim *s, uint64_t seed) {
  s->rs = 1;
  s->rs_seed = seed;
  if (!s->B) s->B = (double *)calloc((size_t)2 * Q * s->n, sizeof(double));
}

#define B_AT(s, a, i, c) ((s)->B[(((int64_t)(a) * Q + (i)) * (s)->n) + (c)])

/* One time step (Eq. LBE with the sputtering law of Eq. f_P_in). */
static void orc_one_step(orc_sim *s) {
  const int nx = s->nx, ny = s->ny, nz = s->nz, ns = s->ns;
  const int64_t plane = (int64_t)nx * ny;
  const int ubw = UB_W(s);

  /* 1. collision at every fluid cell */
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < s->n; ++c) {
    if (s->mask[c]) continue;
    int z = (int)(c / plane);
    int64_t xy = c % plane;
    if (is_bc(s, z)) {
      int side = (z == 0) ? 0 : 1;
      const double *ub = &s->ubuf_prev[((int64_t)side * plane + xy) * ubw];
      double ux = ub[0], uy = ub[1], uz = ub[2];
      if (side == 0 && s->vel_in) {
        ux = 0.0;
        uy = 0.0;
        uz = s->u_in;
      }
      for (int i = 0; i < Q; ++i) F(s, s->fs, 0, i, c) = feq(i, side == 0 ? s->rho_in : s->rho_out, ux, uy, uz);
      for (int a = 1; a < ns; ++a) {
        double rho_a = (side == 0) ? (a == 1 ? s->c_in : 0.0) : ub[3 + a - 1];
        for (int i = 0; i < Q; ++i) F(s, s->fs, a, i, c) = feq(i, rho_a, ux, uy, uz);
      }
      continue;
    }
    double rho = 0, jx = 0, jy = 0, jz = 0;
    for (int i = 0; i < Q; ++i) {
      double fi = F(s, s->f, 0, i, c);
      rho += fi;
      jx += CX[i] * fi;
      jy += CY[i] * fi;
      jz += CZ[i] * fi;
    }
    double rho_a[3] = {rho, 0, 0};
    double rho_t = rho;
    for (int a = 1; a < ns; ++a) {
      double r = 0;
      for (int i = 0; i < Q; ++i) {
        double fi = F(s, s->f, a, i, c);
        r += fi;
        if (s->bary) {
          jx += CX[i] * fi;
          jy += CY[i] * fi;
          jz += CZ[i] * fi;
        }
      }
      rho_a[a] = r;
      rho_t += r;
    }
    /* carrier velocity, or the barycentric one over all arrays; a body force
     * adds half its acceleration */
    const double rt = s->bary ? rho_t : rho;
    double ux = jx / rt, uy = jy / rt, uz = jz / rt;
    uz += 0.5 * s->gz;
    if (!s->zper && (z == 1 || z == nz - 2)) {
      int side = (z == 1) ? 0 : 1;
      double *ub = &s->ubuf_next[((int64_t)side * plane + xy) * ubw];
      ub[0] = ux;
      ub[1] = uy;
      ub[2] = uz;
      for (int a = 1; a < ns; ++a) ub[3 + a - 1] = rho_a[a];
    }
    for (int a = 0; a < ns; ++a)
      for (int i = 0; i < Q; ++i) {
        double fi = F(s, s->f, a, i, c);
        double w = a == 0 ? s->omega : s->omega_s;
        F(s, s->fs, a, i, c) = fi + w * (feq(i, rho_a[a], ux, uy, uz) - fi);
      }
    if (s->gz != 0.0) {
      /* Guo source term of the carrier, F = (0, 0, rho g) */
      const double Fz = rho * s->gz;
      for (int i = 0; i < Q; ++i) {
        const double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
        F(s, s->fs, 0, i, c) += (1.0 - 0.5 * s->omega) * WQ[i] * (3.0 * (CZ[i] - uz) + 9.0 * cu * CZ[i]) * Fz;
      }
    }
  }

  /* 2. species gathered at every catalytic solid node:
   *    A^a(s) = sum over active j of fs_j^a(s - c_j);
   *    random matrix: B^a(s, k) = sum over active j whose draw is k */
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < s->n; ++c) {
    s->A[c] = 0.0;
    s->A[s->n + c] = 0.0;
    if (s->rs)
      for (int a = 0; a < 2; ++a)
        for (int i = 0; i < Q; ++i) B_AT(s, a, i, c) = 0.0;
    if (!s->mask[c] || s->b[c] == 0 || s->sp_bb) continue;
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / plane);
    const uint32_t am = s->rs ? out_mask(s, c) : 0u;
    for (int a = 1; a < ns; ++a) {
      double acc = 0.0;
      for (int j = 1; j < Q; ++j) {
        int64_t src = nbr(nx, ny, nz, s->zper, x, y, z, j, -1);
        if (src >= 0 && !s->mask[src]) {
          acc += F(s, s->fs, a, j, src);
          if (s->rs) B_AT(s, a - 1, orc_rs_choice(s->rs_seed, c, j, s->step, am), c) += F(s, s->fs, a, j, src);
        }
      }
      s->A[(int64_t)(a - 1) * s->n + c] = acc;
    }
  }

  /* 3. streaming (pull) into every interior fluid cell */
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < s->n; ++c) {
    if (s->mask[c]) continue;
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / plane);
    if (is_bc(s, z)) continue;
    for (int i = 0; i < Q; ++i) {
      int64_t src = (i == 0) ? c : nbr(nx, ny, nz, s->zper, x, y, z, i, -1);
      if (!s->mask[src]) {
        for (int a = 0; a < ns; ++a) F(s, s->f, a, i, c) = storeq(s, a, i, F(s, s->fs, a, i, src));
      } else if (s->mask[src] == 2 || s->sp_bb) {
        /* inert solid: every array bounces back halfway */
        for (int a = 0; a < ns; ++a) F(s, s->f, a, i, c) = storeq(s, a, i, F(s, s->fs, a, opp_of(i), c));
      } else {
        /* carrier: halfway bounce-back of its own population along -c_i */
        F(s, s->f, 0, i, c) = storeq(s, 0, i, F(s, s->fs, 0, opp_of(i), c));
        /* species: sputtering law with S_ij = 1/b(src), or with the random
         * one-hot matrix: what the node gathered for link i */
        const double emR = s->desorb ? 1.0 - s->p * s->pSR : 1.0 - s->pSR;
        if (s->rs) {
          double BR = B_AT(s, 0, i, src), BP = B_AT(s, 1, i, src);
          if (ns > 1) F(s, s->f, 1, i, c) = emR * BR;
          if (ns > 2) F(s, s->f, 2, i, c) = s->p * s->pSR * BR + (1.0 - s->pSP) * BP;
        } else {
          double inv_b = 1.0 / (double)s->b[src];
          double AR = s->A[src], AP = s->A[s->n + src];
          if (ns > 1) F(s, s->f, 1, i, c) = emR * AR * inv_b;
          if (ns > 2) F(s, s->f, 2, i, c) = (s->p * s->pSR * AR + (1.0 - s->pSP) * AP) * inv_b;
        }
      }
    }
  }

  /* 4. bookkeeping: wall hits, face fluxes (values as stored) */
  for (int a = 1; a < ns; ++a) {
    double acc = 0.0;
    for (int64_t c = 0; c < s->n; ++c) acc += s->A[(int64_t)(a - 1) * s->n + c];
    s->A_cum[a - 1] += acc;
  }
  if (!s->zper) {
    for (int a = 0; a < ns; ++a) {
      double fin = 0.0, fout = 0.0;
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          int64_t c0 = cidx(s, x, y, 0), c1 = cidx(s, x, y, 1);
          int64_t d1 = cidx(s, x, y, nz - 2), d0 = cidx(s, x, y, nz - 1);
          for (int i = 1; i < Q; ++i) {
            if (CZ[i] == 1) {
              int64_t t0 = nbr(nx, ny, nz, 0, x, y, 0, i, +1);
              if (!s->mask[c0] && !s->mask[t0]) fin += storeq(s, a, i, F(s, s->fs, a, i, c0));
              int64_t t1 = nbr(nx, ny, nz, 0, x, y, nz - 2, i, +1);
              if (!s->mask[d1] && !s->mask[t1]) fout += storeq(s, a, i, F(s, s->fs, a, i, d1));
            } else if (CZ[i] == -1) {
              int64_t t0 = nbr(nx, ny, nz, 0, x, y, 1, i, +1);
              if (!s->mask[c1] && !s->mask[t0]) fin -= storeq(s, a, i, F(s, s->fs, a, i, c1));
              int64_t t1 = nbr(nx, ny, nz, 0, x, y, nz - 1, i, +1);
              if (!s->mask[d0] && !s->mask[t1]) fout -= storeq(s, a, i, F(s, s->fs, a, i, d0));
            }
          }
        }
      s->F_in[a] += fin;
      s->F_out[a] += fout;
    }
  }
  double *t = s->ubuf_prev;
  s->ubuf_prev = s->ubuf_next;
  s->ubuf_next = t;
  s->step += 1;
}

void orc_step(orc_sim *s, int64_t nsteps) {
  for (int64_t k = 0; k < nsteps; ++k) orc_one_step(s);
}

int64_t orc_get_step(const orc_sim *s) { return s->step; }

/* Macroscopic fields at time t: rho of every species array, then the
 * velocity (the carrier's, or the barycentric one when orc_set_barycentric
 * is on; plus g/2 along z under a body force), each [n] (zero at solid
 * cells). out: [ns + 3][n]. */
void orc_fields(const orc_sim *s, double *out) {
  int64_t n = s->n;
  for (int64_t c = 0; c < n; ++c) {
    for (int k = 0; k < s->ns + 3; ++k) out[(int64_t)k * n + c] = 0.0;
    if (s->mask[c]) continue;
    double jx = 0, jy = 0, jz = 0, rho_t = 0;
    for (int a = 0; a < s->ns; ++a) {
      double r = 0;
      for (int i = 0; i < Q; ++i) {
        double fi = F(s, s->f, a, i, c);
        r += fi;
        if (a == 0 || s->bary) {
          jx += CX[i] * fi;
          jy += CY[i] * fi;
          jz += CZ[i] * fi;
        }
      }
      out[(int64_t)a * n + c] = r;
      rho_t += r;
    }
    double rho = s->bary ? rho_t : out[c];
    out[(int64_t)(s->ns + 0) * n + c] = jx / rho;
    out[(int64_t)(s->ns + 1) * n + c] = jy / rho;
    out[(int64_t)(s->ns + 2) * n + c] = jz / rho + 0.5 * s->gz;
  }
}

/* Observables at time t (FP64):
 *   scal[0..2]  interior masses M_C, M_R, M_P (planes 1..nz-2, or all planes
 *               in a z-periodic box)
 *   scal[3]     eta = sum_xy rho_P(z = nz-2) / sum_xy rho_R(z = 1)   (Eq. eff)
 *   scal[4..6]  cumulative inflow through the inlet face (C, R, P)
 *   scal[7..9]  cumulative outflow through the outlet face (C, R, P)
 *   scal[10,11] cumulative wall hits sum A^R, sum A^P
 *   scal[12]    reacted  = p pS_R sum A^R
 *   scal[13]    stuck R  = pS_R (1 - p) sum A^R (0 when the stuck R desorbs)
 *   scal[14]    stuck P  = pS_P sum A^P
 *   scal[15]    carrier mass residual  M_C - M_C0 - (in - out)
 *   scal[16]    R+P mass residual      M_RP - M_RP0 - (in - out) + stuck
 *               (+ reacted when only R is simulated)
 *   per layer z (each nz long, optional): rho_C, rho_R, rho_P plane sums,
 *               Phi_P(z) = sum rho_P u_z (Eq. Phi_P), reaction rate
 *               p pS_R sum over nodes in the plane of A^R (last step)
 *   site (optional, n long): p pS_R A^R(s) at every solid cell (last step) */
void orc_observables(const orc_sim *s, double *scal, double *rhoC_z, double *rhoR_z, double *rhoP_z,
                     double *phiP_z, double *react_z, double *site) {
  int64_t n = s->n, plane = (int64_t)s->nx * s->ny;
  int nz = s->nz;
  double *fld = (double *)malloc(sizeof(double) * n * (s->ns + 3));
  orc_fields(s, fld);
  double M[3] = {0, 0, 0};
  double mRin = 0.0, mPout = 0.0;
  for (int z = 0; z < nz; ++z) {
    double sC = 0, sR = 0, sP = 0, ph = 0, rr = 0;
    /* inlet/outlet planes carry no state of their own: reported as 0 */
    for (int64_t xy = 0; xy < (is_bc(s, z) ? 0 : plane); ++xy) {
      int64_t c = (int64_t)z * plane + xy;
      if (s->mask[c]) {
        if (s->ns > 1) rr += s->p * s->pSR * s->A[c];
        continue;
      }
      sC += fld[c];
      if (s->ns > 1) sR += fld[n + c];
      if (s->ns > 2) {
        sP += fld[2 * n + c];
        ph += fld[2 * n + c] * fld[(int64_t)(s->ns + 2) * n + c];
      }
    }
    if (rhoC_z) rhoC_z[z] = sC;
    if (rhoR_z) rhoR_z[z] = sR;
    if (rhoP_z) rhoP_z[z] = sP;
    if (phiP_z) phiP_z[z] = ph;
    if (react_z) react_z[z] = rr;
    if (!is_bc(s, z)) {
      M[0] += sC;
      M[1] += sR;
      M[2] += sP;
    }
    if (z == 1) mRin = sR;
    if (z == nz - 2) mPout = sP;
  }
  scal[0] = M[0];
  scal[1] = M[1];
  scal[2] = M[2];
  scal[3] = (mRin != 0.0) ? mPout / mRin : 0.0;
  for (int a = 0; a < 3; ++a) {
    scal[4 + a] = s->F_in[a];
    scal[7 + a] = s->F_out[a];
  }
  scal[10] = s->A_cum[0];
  scal[11] = s->A_cum[1];
  scal[12] = s->p * s->pSR * s->A_cum[0];
  scal[13] = s->desorb ? 0.0 : s->pSR * (1.0 - s->p) * s->A_cum[0];
  scal[14] = s->pSP * s->A_cum[1];
  scal[15] = M[0] - s->M0[0] - (s->F_in[0] - s->F_out[0]);
  scal[16] = (M[1] + M[2]) - (s->M0[1] + s->M0[2]) - (s->F_in[1] + s->F_in[2] - s->F_out[1] - s->F_out[2]) +
             scal[13] + scal[14] + (s->ns == 2 ? scal[12] : 0.0); /* R only: reacted R leaves */
  if (site) {
    for (int64_t c = 0; c < n; ++c) site[c] = (s->mask[c] && s->ns > 1) ? s->p * s->pSR * s->A[c] : 0.0;
  }
  free(fld);
}
