// Fused collide-stream-boundary kernel and state readers, templated on the
// population storage. Included once per storage type (step_f32.cu,
// step_f16.cu, step_bf16.cu) so the three compile in parallel.
//
// Time stepping follows the lattice BGK equation of the paper's Appendix
// (Eq. LBE, Eq. feq, one omega for every species), with species relaxed
// towards an equilibrium built on the carrier velocity, halfway bounce-back
// of the carrier at solid links, and the sputtering law (Appendix,
// Eq. f_P_in) with S_ij = 1/b(x) at catalytic nodes.
//
// Streaming is in place (AA pattern): one population array. An even step
// reads a cell's own slots f[i][x], collides, and writes f*_i to f[opp(i)][x];
// an odd step reads f[opp(i)][x - c_i] (the neighbour's even-step output),
// collides, and writes f*_i to f[i][x + c_i]. After an odd step the array
// holds the streamed populations in natural order again.
//   - carrier, solid upwind (x - c_i solid): the slot the cell itself wrote
//     for the reversed direction holds f*_opp(i)(x) -> halfway bounce-back;
//   - species, solid target (x + c_i solid): f*_i is added to the node's
//     accumulator A_cur (this step); species, solid upwind: the population is
//     rebuilt from the node's accumulator of the previous step, A_prev, by the
//     sputtering law. So the wall re-emits one step after the hit, the same
//     timing as bounce-back, with no grid-wide synchronisation. A 3-deep ring
//     (prev, cur, next) lets every step clear the buffer of the step after.
//   - inlet plane z=0 / outlet plane z=nz-1: equilibrium with the velocity of
//     plane 1 / nz-2 from the previous step (and, at the outlet, the species
//     densities of plane nz-2), passed through a double-buffered plane cache.
//
// All arithmetic is on the stored scaled deviations d_i = (f_i - w_i rho_ref)
// / w_i (rho_ref = 1 for the carrier, 0 for the species): drho = sum w d,
// j = sum w c d (the w_i rho_ref parts cancel since sum w c = 0),
// rho = rho_ref + drho, u = j / rho, and the equilibrium in the same units,
// deq_i = (rho - rho_ref) + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2) (carrier) or
// rho_s + rho_s (3 c.u + 4.5 (c.u)^2 - 1.5 u^2) (species), so that
// d*_i = d_i + omega (deq_i - d_i).
#pragma once

#include "lbm_internal.h"

namespace lbm {

// Neighbour cells of one cell (32-bit: boxes hold fewer than 2^31 cells).
struct Nbr {
  int32_t cell, oxm, oxp, oym, oyp, ozm, ozp;
  __device__ __forceinline__ Nbr(int32_t c, int x, int y, int z, int nx, int ny, int nz, int per_z) {
    const int32_t plane = nx * ny;
    cell = c;
    oxm = (x == 0) ? nx - 1 : -1;
    oxp = (x == nx - 1) ? -(nx - 1) : 1;
    oym = ((y == 0) ? ny - 1 : -1) * nx;
    oyp = ((y == ny - 1) ? -(ny - 1) : 1) * nx;
    ozm = -plane;
    ozp = plane;
    if (per_z) {
      if (z == 0) ozm = (nz - 1) * plane;
      if (z == nz - 1) ozp = -(nz - 1) * plane;
    }
  }
  __device__ __forceinline__ int32_t at(int dx, int dy, int dz) const {
    return cell + (dx < 0 ? oxm : (dx > 0 ? oxp : 0)) + (dy < 0 ? oym : (dy > 0 ? oyp : 0)) +
           (dz < 0 ? ozm : (dz > 0 ? ozp : 0));
  }
};

// Population layout: warp-blocked structure of arrays. Entry e, species
// array s, direction i lives at ((e / 32) * NS * 19 + s * 19 + i) * 32 + e % 32:
// a warp's 32 consecutive entries are contiguous for every (s, i), and all
// (s, i) of one entry are compile-time offsets from one base.
template <int NS>
__device__ __forceinline__ int64_t ent_base(int32_t e) {
  return (int64_t)(e >> 5) * (NS * kQ * 32) + (e & 31);
}
__device__ __forceinline__ constexpr int si_off(int s, int i) { return (s * kQ + i) * 32; }
// ent_base modulo 2^32: the difference of two of these is the exact element
// distance between two entries whenever that distance is below 2^31
template <int NS>
__device__ __forceinline__ uint32_t ent_base32(int32_t e) {
  return (uint32_t)e + ((uint32_t)e >> 5) * (uint32_t)(NS * kQ * 32 - 32);
}

// Population loads name their cache operator (ld.global.ca): never the
// non-coherent read-only path, which a const __restrict__ pointer would
// allow. Within one multi-step batched launch a CTA reads populations that
// other CTAs wrote earlier in the same launch; ordinary loads observe them
// after the step-ordering acquire, non-coherent loads need not.
template <typename T>
__device__ __forceinline__ T ld_pop(const T *p) {
  return __ldca(p);
}
// Population stores are streaming stores (st.global.cs): each stored value
// is read once, by the next step. Measured 1-2% faster per step than plain
// stores; coherence is unchanged, so the multi-step batched launch may use
// them too.

template <int LAYOUT>
__device__ __forceinline__ int32_t lat_of(const StepArgs &a, int32_t cell) {
  if (LAYOUT == LBM_LAYOUT_DENSE) return cell;
  return __ldg(a.idx + LBM_OFF(a, kChkIdx, 0, cell, LBM_NCELLS(a)));
}

// Wall hits of the previous step at node k, species row sp (0 R, 1 P): the
// node's total, or, under the random sputtering matrix, the sum over its
// link slots. And what the node re-emits along its outgoing link i: a share
// of the hits times 1/b (uniform matrix) or the link's own slot, whose rank
// is the number of active links below i (random matrix, factor 1).
template <bool DET>
__device__ __forceinline__ double hits_d(const StepArgs &a, int sp, int64_t k) {
  if (!a.rs) return acc_get_d<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, sp * a.acc_row + k, LBM_NACC(a)));
  double h = 0.0;
  for (int32_t l = __ldg(a.node_off + LBM_OFF(a, kChkNode, 0, k, a.n_nodes + 1));
       l < __ldg(a.node_off + LBM_OFF(a, kChkNode, 0, k + 1, a.n_nodes + 1)); ++l)
    h += acc_get_d<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, sp * a.acc_row + l, LBM_NACC(a)));
  return h;
}
// (rs: the random matrix, fixed at compile time on the step path; the
// observables' readers pass the simulation's runtime flag)
__device__ __forceinline__ int64_t emit_index(bool rs, const StepArgs &a, int i, int32_t node, int32_t node_cell) {
  if (!rs) return (int64_t)node;
  return (int64_t)__ldg(a.node_off + LBM_OFF(a, kChkNode, 0, node, a.n_nodes + 1)) +
         __popc(__ldg(a.cell_bits + LBM_OFF(a, kChkIdx, 0, node_cell, LBM_NCELLS(a))) & ((1u << i) - 1u));
}
__device__ __forceinline__ float emit_scale(bool rs, const StepArgs &a, int32_t node) {
  return rs ? 1.0f : __ldg(a.inv_b + LBM_OFF(a, kChkNode, 0, node, a.n_nodes));
}
// Index of the accumulator that the species population arriving at node
// `node` (in cell node_cell) along c_j adds to, species row sp.
template <bool RS>
__device__ __forceinline__ int64_t hit_index(const StepArgs &a, int sp, int32_t node, int32_t node_cell, int j,
                                             int64_t t) {
  if (!RS) return sp * a.acc_row + node;
  const int32_t o = __ldg(a.node_off + LBM_OFF(a, kChkNode, 0, node, a.n_nodes + 1));
  return sp * a.acc_row + o +
         rs_rank(a.rs_key, node_cell, j, t, __ldg(a.node_off + LBM_OFF(a, kChkNode, 0, node + 1, a.n_nodes + 1)) - o);
}

// Populations of lattice entry L at the current time as deviations
// g = f - w rho_ref, as a two-lattice scheme would hold them (natural
// order), for a state of parity ODD (ODD = 1: the last completed step was
// an even one).
template <int ST, int LAYOUT, int NS, int ODD, bool DET>
__device__ __forceinline__ void load_cell(const StepArgs &a, int32_t L, const Nbr &nb, uint32_t nbm,
                                          float (&f)[NS][kQ]) {
  using S = Store<ST>;
  using T = typename S::T;
  const T *F = static_cast<const T *>(a.f);
  const int64_t own = ent_base<NS>(L);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const bool solid_up = (i != 0) && ((nbm >> opp(i)) & 1u);
    if (!solid_up) {
      int64_t base = own;
      int slot = i;
      if (ODD && i != 0) {
        base = ent_base<NS>(lat_of<LAYOUT>(a, nb.at(-cx(i), -cy(i), -cz(i))));
        slot = opp(i);
      }
#pragma unroll
      for (int s = 0; s < NS; ++s)
        f[s][i] = wq(i) * S::load(ld_pop(F + LBM_OFF(a, kChkPop, 0, base + si_off(s, slot), LBM_NPOP(a, NS))), s);
    } else {
      // carrier: the cell's own reversed post-collision population sits in
      // slot i in both parities (written by the previous odd step as the
      // bounce-back of its outgoing opp(i), or by the even step at opp(opp(i)))
      f[0][i] = wq(i) * S::load(ld_pop(F + LBM_OFF(a, kChkPop, 0, own + si_off(0, i), LBM_NPOP(a, NS))), 0);
      const int32_t node_cell = nb.at(-cx(i), -cy(i), -cz(i));
      const int32_t node = __ldg(a.idx + LBM_OFF(a, kChkIdx, 0, node_cell, LBM_NCELLS(a)));
      if (NS > 1 && (node < 0 || a.sp_bb)) {
        // inert solid: every array's own reversed population, as the carrier's
#pragma unroll
        for (int s = 1; s < NS; ++s)
          f[s][i] = wq(i) * S::load(ld_pop(F + LBM_OFF(a, kChkPop, 0, own + si_off(s, i), LBM_NPOP(a, NS))), s);
      } else if (NS > 1) {
        const float ib = emit_scale(a.rs != 0, a, node);
        const int64_t e = emit_index(a.rs != 0, a, i, node, node_cell);
        const float AR = acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, e, LBM_NACC(a)));
        f[1][i] = a.em_R * AR * ib;
        if (NS > 2) {
          const float AP = acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, a.acc_row + e, LBM_NACC(a)));
          f[2][i] = (a.em_PR * AR + a.em_P * AP) * ib;
        }
      }
    }
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide FP64 sum of K per-thread values, fixed order; result valid in
// thread 0. Must be called by every thread of the block.
template <int K, typename V>
__device__ __forceinline__ void block_sum_d(const V (&v)[K], double (&out)[K]) {
  __shared__ double sh[K][kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = warp_sum_d((double)v[k]);
    if (lane == 0) sh[k][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = (lane < kBlock / 32) ? sh[k][lane] : 0.0;
      s = warp_sum_d(s);
      if (lane == 0) out[k] = s;
    }
  }
  __syncthreads();
}

// Gathered populations of one species array (scaled deviations d) for
// lattice entry L. nl[k] (odd steps, fluid-only layout) holds idx[cell + c_k]:
// the neighbour's lattice entry when it is fluid, its node number when solid.
// FAST: the whole warp has no solid neighbour, so no link needs a
// substitution.
template <int ST, int LAYOUT, int NS, int ODD, bool DET, int SP, bool FAST, bool RS, int PHYS>
__device__ __forceinline__ void load_species(const StepArgs &a, int32_t L, const Nbr &nb, uint32_t nbm,
                                             const int32_t (&nl)[kQ], float (&d)[kQ]) {
  using S = Store<ST>;
  using T = typename S::T;
  const T *F = static_cast<const T *>(a.f);
  const T *own = F + ent_base<NS>(L);
  // every population load first (a solid upwind link reads a harmless
  // in-bounds slot that is replaced below), substitutions after
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const bool solid_up = !FAST && (i != 0) && ((nbm >> opp(i)) & 1u);
    if (ODD && i != 0 && !solid_up) {
      if (FAST && LAYOUT != LBM_LAYOUT_DENSE) {
        // nl holds element offsets from the entry's own base on this path
        d[i] = S::load(ld_pop(own + LBM_OFF(a, kChkPop, own - F, nl[opp(i)] + si_off(SP, opp(i)), LBM_NPOP(a, NS))),
                       SP);
      } else {
        const int32_t src = (LAYOUT == LBM_LAYOUT_DENSE) ? nb.at(-cx(i), -cy(i), -cz(i)) : nl[opp(i)];
        d[i] = S::load(ld_pop(F + LBM_OFF(a, kChkPop, 0, ent_base<NS>(src) + si_off(SP, opp(i)), LBM_NPOP(a, NS))),
                       SP);
      }
    } else {
      d[i] = S::load(ld_pop(own + LBM_OFF(a, kChkPop, own - F, si_off(SP, i), LBM_NPOP(a, NS))), SP);
    }
  }
  if (!FAST && SP > 0 && nbm) {
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      if ((nbm >> opp(i)) & 1u) {
        const int32_t node =
            (ODD && LAYOUT != LBM_LAYOUT_DENSE)
                ? nl[opp(i)]
                : __ldg(a.idx + LBM_OFF(a, kChkIdx, 0, nb.at(-cx(i), -cy(i), -cz(i)), LBM_NCELLS(a)));
        // inert solid (or species bounce-back): the own slot holds the bounce-back
        if (PHYS == kPhysChannel && (node < 0 || a.sp_bb)) continue;
        const float ib = emit_scale(RS, a, node) * inv_wq(i);
        const int64_t e = emit_index(RS, a, i, node, RS ? nb.at(-cx(i), -cy(i), -cz(i)) : 0);
        const float AR = acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, e, LBM_NACC(a)));
        if (SP == 1) {
          d[i] = a.em_R * AR * ib;
        } else {
          const float AP = acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, a.acc_row + e, LBM_NACC(a)));
          d[i] = (a.em_PR * AR + a.em_P * AP) * ib;
        }
      }
    }
  }
}

// Store the post-collision populations of one species array, account the
// inlet/outlet face flows (fsel: 0 inlet plane, 1 plane 1, 2 plane nz-2,
// 3 outlet plane, -1 elsewhere) and send species that hit catalytic nodes
// to this step's accumulators.
template <int ST, int LAYOUT, int NS, int ODD, bool DET, int SP, bool FAST, bool RS, int PHYS>
__device__ __forceinline__ void store_species(const StepArgs &a, int32_t L, const Nbr &nb, uint32_t nbm,
                                              const int32_t (&nl)[kQ], const float (&d)[kQ], bool bc, int z,
                                              int fsel, int64_t t, float (&flux)[6]) {
  // per-cell random word of the stochastic rounding (16-bit storage only)
  const uint32_t rh = (ST == LBM_FP32) ? 0u : mix32((uint32_t)L ^ step_seed_of(t, a.seed_mix));
  using S = Store<ST>;
  using T = typename S::T;
  T *__restrict__ F = static_cast<T *>(a.f);
  T *own = F + ent_base<NS>(L);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const bool solid_dn = !FAST && (i != 0) && ((nbm >> i) & 1u);
    const bool outside = !FAST && bc && ((z == 0 && cz(i) < 0) || (z == a.nz - 1 && cz(i) > 0));
    const T q = S::store(d[i], SP, sr_bits(rh, SP, i));
    if (!FAST && fsel >= 0 && !solid_dn && !outside) {
      const bool up = cz(i) > 0, dn = cz(i) < 0;
      const float sgn = ((fsel == 0 || fsel == 2) && up) ? 1.f : (((fsel == 1 || fsel == 3) && dn) ? -1.f : 0.f);
      if (sgn != 0.f) flux[(fsel <= 1 ? 0 : 3) + SP] += sgn * wq(i) * S::load(q, SP);
    }
    if (SP > 0 && solid_dn) {
      const int32_t node_cell = nb.at(cx(i), cy(i), cz(i));
      const int32_t node = (ODD && LAYOUT != LBM_LAYOUT_DENSE)
                               ? nl[i]
                               : __ldg(a.idx + LBM_OFF(a, kChkIdx, 0, node_cell, LBM_NCELLS(a)));
      if (PHYS != kPhysChannel || (node >= 0 && !a.sp_bb)) {
        acc_add<DET>(a.A_cur, LBM_OFF(a, kChkAcc, 0, hit_index<RS>(a, SP - 1, node, node_cell, i, t), LBM_NACC(a)),
                     wq(i) * d[i]);
        continue;
      }
      // inert solid: bounce back below, as the carrier does
    }
    if (!ODD) {
      __stcs(&own[LBM_OFF(a, kChkPop, own - F, si_off(SP, opp(i)), LBM_NPOP(a, NS))], q);
    } else if (i == 0) {
      __stcs(&own[LBM_OFF(a, kChkPop, own - F, si_off(SP, 0), LBM_NPOP(a, NS))], q);
    } else if (solid_dn) {
      // carrier and inert walls: halfway bounce-back slot
      __stcs(&own[LBM_OFF(a, kChkPop, own - F, si_off(SP, opp(i)), LBM_NPOP(a, NS))], q);
    } else if (!outside) {
      if (FAST && LAYOUT != LBM_LAYOUT_DENSE) {
        __stcs(&own[LBM_OFF(a, kChkPop, own - F, nl[i] + si_off(SP, i), LBM_NPOP(a, NS))], q);
      } else {
        const int32_t t = (LAYOUT == LBM_LAYOUT_DENSE) ? nb.at(cx(i), cy(i), cz(i)) : nl[i];
        __stcs(&F[LBM_OFF(a, kChkPop, 0, ent_base<NS>(t) + si_off(SP, i), LBM_NPOP(a, NS))], q);
      }
    }
  }
}

// Species phase: gather, relax towards feq(rho_s, u) with the cell's
// velocity u (or the inlet/outlet equilibrium), store.
template <int ST, int LAYOUT, int NS, int ODD, bool DET, int SP, bool FAST, bool RS, int PHYS>
__device__ __forceinline__ void species_phase(const StepArgs &a, int32_t L, const Nbr &nb, uint32_t nbm,
                                              const int32_t (&nl)[kQ], float ux, float uy, float uz, bool bc,
                                              int z, int32_t xy, int32_t plane, int fsel, int64_t t,
                                              float (&flux)[6]) {
  float d[kQ];
  float rs;
  if (FAST || !bc) {
    load_species<ST, LAYOUT, NS, ODD, DET, SP, FAST, RS, PHYS>(a, L, nb, nbm, nl, d);
    rs = 0.f;
#pragma unroll
    for (int i = 0; i < kQ; ++i) rs += wq(i) * d[i];
    if (!FAST && !a.periodic_z && (z == 1 || z == a.nz - 2))
      a.ub_cur[LBM_OFF(a, kChkUb, 0, (int64_t)((z == 1 ? 0 : 5) + 2 + SP) * plane + xy, LBM_NUB(a))] = rs;
  } else {
    rs = (z == 0) ? (SP == 1 ? a.c_in : 0.0f)
                  : a.ub_prev[LBM_OFF(a, kChkUb, 0, (int64_t)(5 + 2 + SP) * plane + xy, LBM_NUB(a))];
  }
  const float u2 = 1.5f * (ux * ux + uy * uy + uz * uz);
  const bool eq = !FAST && bc;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float cu = 3.0f * (cx(i) * ux + cy(i) * uy + cz(i) * uz);
    // rho_s + rho_s P rather than rho_s (1 + P): the rounding then scales with
    // P (~1e-3), so sum w deq stays rho_s to FP32 precision (mass conservation)
    const float deq = fmaf(rs, cu + 0.5f * cu * cu - u2, rs);
    d[i] = eq ? deq : d[i] + (PHYS == kPhysCarrier ? a.omega : a.omega_s) * (deq - d[i]);
  }
  store_species<ST, LAYOUT, NS, ODD, DET, SP, FAST, RS, PHYS>(a, L, nb, nbm, nl, d, bc, z, fsel, t, flux);
}

// Adds the mass and momentum of one species array (gathered as in its own
// phase) to m = (rho, jx, jy, jz).
template <int ST, int LAYOUT, int NS, int ODD, bool DET, int SP, bool FAST, bool RS, int PHYS>
__device__ __forceinline__ void add_species_moments(const StepArgs &a, int32_t L, const Nbr &nb, uint32_t nbm,
                                                    const int32_t (&nl)[kQ], float (&m)[4]) {
  float d[kQ];
  load_species<ST, LAYOUT, NS, ODD, DET, SP, FAST, RS, PHYS>(a, L, nb, nbm, nl, d);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float wd = wq(i) * d[i];
    m[0] += wd;
    m[1] += cx(i) * wd;
    m[2] += cy(i) * wd;
    m[3] += cz(i) * wd;
  }
}

// Update of one cell: carrier (moments, BGK or inlet/outlet equilibrium,
// store), then each species. u is the carrier's velocity, or with BARY the
// barycentric velocity sum_a j_a / sum_a rho_a over every array (Appendix,
// velocity equation): the species arrays are then gathered once for their
// moments before the carrier and again in their own phase (the second
// gather reads the same addresses and mostly hits L1). Only one species
// array is live in registers at a time.
template <int ST, int LAYOUT, int NS, int ODD, bool DET, bool FAST, bool RS, int PHYS>
__device__ __forceinline__ void cell_update(const StepArgs &a, int32_t L, int32_t cell, uint32_t nbm, int64_t t,
                                            float (&flux)[6]) {
  const int32_t plane = a.nx * a.ny;
  const int z = cell / plane;
  const int32_t xy = cell - z * plane;
  const int y = xy / a.nx;
  const int x = xy - y * a.nx;
  const Nbr nb(cell, x, y, z, a.nx, a.ny, a.nz, a.periodic_z);
  const bool open = !a.periodic_z;
  const bool bc = !FAST && open && (z == 0 || z == a.nz - 1);
  const int fsel =
      (FAST || !open) ? -1 : (z == 0 ? 0 : (z == 1 ? 1 : (z == a.nz - 2 ? 2 : (z == a.nz - 1 ? 3 : -1))));

  // odd steps, fluid-only addressing: the neighbour entries idx[cell + c_k]
  // (fluid neighbours) or node numbers (solid ones); on the fast path, where
  // every neighbour is fluid and within two planes, their element offsets
  // from this entry's own base instead (32-bit, so each gather and scatter
  // takes a single address operation)
  int32_t nl[kQ];
  if (ODD && LAYOUT != LBM_LAYOUT_DENSE) {
    const uint32_t own32 = ent_base32<NS>(L);
    nl[0] = FAST ? 0 : L;
#pragma unroll
    for (int k = 1; k < kQ; ++k) {
      const bool out = bc && ((z == 0 && cz(k) < 0) || (z == a.nz - 1 && cz(k) > 0));
      const int32_t e = out ? L : __ldg(a.idx + LBM_OFF(a, kChkIdx, 0, nb.at(cx(k), cy(k), cz(k)), LBM_NCELLS(a)));
      nl[k] = FAST ? (int32_t)(ent_base32<NS>(e) - own32) : e;
    }
  }

  constexpr bool BARY = PHYS == kPhysBary;
  float ms[4] = {0.f, 0.f, 0.f, 0.f};  // species rho, jx, jy, jz (BARY)
  if (BARY && !bc) {
    add_species_moments<ST, LAYOUT, NS, ODD, DET, 1, FAST, RS, PHYS>(a, L, nb, nbm, nl, ms);
    if (NS > 2) add_species_moments<ST, LAYOUT, NS, ODD, DET, 2, FAST, RS, PHYS>(a, L, nb, nbm, nl, ms);
  }

  float ux, uy, uz;
  {
    float d[kQ];
    float drho;
    if (!bc) {
      load_species<ST, LAYOUT, NS, ODD, DET, 0, FAST, RS, PHYS>(a, L, nb, nbm, nl, d);
      float jx = 0.f, jy = 0.f, jz = 0.f;
      drho = 0.f;
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const float wd = wq(i) * d[i];
        drho += wd;
        jx += cx(i) * wd;
        jy += cy(i) * wd;
        jz += cz(i) * wd;
      }
      const float inv_rho = 1.0f / (BARY ? (1.0f + drho) + ms[0] : 1.0f + drho);
      ux = (BARY ? jx + ms[1] : jx) * inv_rho;
      uy = (BARY ? jy + ms[2] : jy) * inv_rho;
      uz = (BARY ? jz + ms[3] : jz) * inv_rho;
      if (PHYS == kPhysChannel) uz += 0.5f * a.g_z;  // body force: the velocity half a step on
      if (!FAST && open && (z == 1 || z == a.nz - 2)) {
        // (u_x, u_y, u_z at ub[0], ub[plane], ub[2 plane]: the check bounds the last)
        float *ub = a.ub_cur + LBM_OFF(a, kChkUb, 0, (int64_t)(z == 1 ? 0 : 5) * plane + xy,
                                       LBM_NUB(a) - 2 * (int64_t)plane);
        ub[0] = ux;
        ub[plane] = uy;
        ub[2 * (int64_t)plane] = uz;
      }
    } else {
      const float *ub = a.ub_prev + LBM_OFF(a, kChkUb, 0, (int64_t)(z == 0 ? 0 : 5) * plane + xy,
                                            LBM_NUB(a) - 2 * (int64_t)plane);
      ux = ub[0];
      uy = ub[plane];
      uz = ub[2 * (int64_t)plane];
      if (z == 0 && a.vel_in) {  // velocity inlet: (0, 0, u_in)
        ux = 0.f;
        uy = 0.f;
        uz = a.u_in;
      }
      drho = (z == 0) ? a.drho_in : a.drho_out;
    }
    const float rho = 1.0f + drho;
    const float u2 = 1.5f * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float cu = 3.0f * (cx(i) * ux + cy(i) * uy + cz(i) * uz);
      const float deq = drho + rho * (cu + 0.5f * cu * cu - u2);
      d[i] = bc ? deq : d[i] + a.omega * (deq - d[i]);
    }
    if (PHYS == kPhysChannel && !bc && a.g_z != 0.f) {
      // body force F = rho g along z, Guo, Zheng and Shi (2002): in scaled
      // deviations the source adds (1 - omega/2) [3 (c_iz - u_z) + 9 (c_i . u) c_iz] F_z
      const float fz = (1.0f - 0.5f * a.omega) * rho * a.g_z;
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const float cu = 3.0f * (cx(i) * ux + cy(i) * uy + cz(i) * uz);
        d[i] = fmaf(fz, 3.0f * (cz(i) - uz) + cu * (3.0f * cz(i)), d[i]);
      }
    }
    store_species<ST, LAYOUT, NS, ODD, DET, 0, FAST, RS, PHYS>(a, L, nb, nbm, nl, d, bc, z, fsel, t, flux);
  }
  if (NS > 1)
    species_phase<ST, LAYOUT, NS, ODD, DET, 1, FAST, RS, PHYS>(a, L, nb, nbm, nl, ux, uy, uz, bc, z, xy, plane, fsel, t,
                                                      flux);
  if (NS > 2)
    species_phase<ST, LAYOUT, NS, ODD, DET, 2, FAST, RS, PHYS>(a, L, nb, nbm, nl, ux, uy, uz, bc, z, xy, plane, fsel, t,
                                                      flux);
}

// One time step: one thread per lattice entry, plus the catalytic-node pass
// and the per-block face-flow bookkeeping.
template <int ST, int LAYOUT, int NS, int ODD, bool DET, bool RS, int PHYS>
__device__ __forceinline__ void step_block(const StepArgs &a, const int blk, const int64_t t) {
  const int32_t L = (int32_t)(blk * kBlock + threadIdx.x);
  const int32_t plane = a.nx * a.ny;
  float flux[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // in C,R,P ; out C,R,P

  bool live = L < a.n_lat;
  int32_t cell = 0;
  uint32_t nbm = 0;
  if (live) {
    cell = (LAYOUT == LBM_LAYOUT_DENSE) ? L : __ldg(a.fcell + L);
    if (LAYOUT == LBM_LAYOUT_DENSE && __ldg(a.mask + cell)) live = false;
    nbm = __ldg(a.nbm + L);
  }
  // warp-uniform fast path: no solid neighbour and away from the planes
  // z = 0, 1, nz-2, nz-1 that take part in the inlet/outlet conditions
  const int zc = cell / plane;
  // (periodic z: the wrapping planes 0 and nz-1 are left to the general path,
  // so that fast-path neighbours lie within two planes)
  const bool plain =
      !live || (nbm == 0 && (a.periodic_z ? (zc > 0 && zc < a.nz - 1) : (zc > 1 && zc < a.nz - 2)));
  if (__all_sync(0xffffffffu, plain)) {
    if (live) cell_update<ST, LAYOUT, NS, ODD, DET, true, RS, PHYS>(a, L, cell, 0u, t, flux);
  } else if (live) {
    cell_update<ST, LAYOUT, NS, ODD, DET, false, RS, PHYS>(a, L, cell, nbm, t, flux);
  }

  // catalytic-node pass: bank the previous step's wall hits, clear the next buffer
  if ((int64_t)blk * kBlock < a.n_nodes) {
    float hv[2] = {0.f, 0.f};
    if (L < a.n_nodes) {
      if (RS) {
        for (int32_t k = __ldg(a.node_off + LBM_OFF(a, kChkNode, 0, L, a.n_nodes + 1));
             k < __ldg(a.node_off + LBM_OFF(a, kChkNode, 0, L + 1, a.n_nodes + 1)); ++k) {
          hv[0] += acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, k, LBM_NACC(a)));
          acc_clear<DET>(a.A_next, LBM_OFF(a, kChkAcc, 0, k, LBM_NACC(a)));
          if (NS > 2) {
            hv[1] += acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, a.acc_row + k, LBM_NACC(a)));
            acc_clear<DET>(a.A_next, LBM_OFF(a, kChkAcc, 0, a.acc_row + k, LBM_NACC(a)));
          }
        }
      } else {
        hv[0] = acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, L, LBM_NACC(a)));
        acc_clear<DET>(a.A_next, LBM_OFF(a, kChkAcc, 0, L, LBM_NACC(a)));
        if (NS > 2) {
          hv[1] = acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, a.acc_row + L, LBM_NACC(a)));
          acc_clear<DET>(a.A_next, LBM_OFF(a, kChkAcc, 0, a.acc_row + L, LBM_NACC(a)));
        }
      }
    }
    double hs[2];
    block_sum_d<2>(hv, hs);
    if (threadIdx.x == 0) {
      a.node_cum[2 * (int64_t)blk + 0] += hs[0];
      a.node_cum[2 * (int64_t)blk + 1] += hs[1];
    }
  }
  // inlet / outlet face flows
  if (!a.periodic_z) {
    const int b = blk;
    int slot = -1;
    if (b < a.n_lo_blocks)
      slot = b;
    else if (b >= a.hi_base && b < a.n_lat_blocks)
      slot = a.n_lo_blocks + (b - a.hi_base);
    if (slot >= 0) {
      double fs[6];
      block_sum_d<6>(flux, fs);
      if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) a.flux_cum[6 * (int64_t)slot + k] += fs[k];
      }
    }
  }
}

template <int ST, int LAYOUT, int NS, int ODD, bool DET, bool RS, int PHYS>
__global__ void __launch_bounds__(kBlock, ODD ? kOddMinBlocks : kStepMinBlocks) step_kernel(const StepArgs a) {
  step_block<ST, LAYOUT, NS, ODD, DET, RS, PHYS>(a, (int)blockIdx.x, a.t);
}

// Batched launch advancing many simulations by several steps (continuous
// batching). Work block w of a step belongs to the simulation k with
// block_start[k] <= w < block_start[k + 1], whose arguments (constant bank)
// and own parity pick the path.
__device__ __forceinline__ int batch_sim_of(const BatchLaunch &p, int w) {
  int lo = 0, hi = p.n_sims - 1;  // last simulation with block_start <= w
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.block_start[mid] <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// One launch covers p.n_steps steps: n_steps x total_blocks CTAs, one work
// block each. With several steps, a CTA takes the next ticket when it starts
// (ticket = step x total_blocks + work block), and a CTA of step k > 0 first
// waits until every work block of step k - 1 has finished: the in-place AA
// update of step k reads what step k - 1 wrote. Tickets follow the order in
// which CTAs actually start, so every CTA a waiter depends on is already
// running or done, and the lowest unfinished step never waits: the launch
// needs no co-residency guarantee. Each CTA runs exactly one work block, with
// no loop around the step (a loop of steps inside one CTA made the compiler
// spill about 1 KB per thread).
template <int ST, int LAYOUT, int NS, bool DET, bool RS, int PHYS>
__global__ void __launch_bounds__(kBlock, kOddMinBlocks) batch_step_kernel(const __grid_constant__ BatchLaunch p) {
  int t = (int)blockIdx.x;
  if (p.n_steps > 1) {
    __shared__ int s_ticket;
    if (threadIdx.x == 0) {
      int tk = (int)atomicAdd(&p.sync->ticket, 1u);
      const int k = tk / p.total_blocks;
      if (*(volatile int *)&p.sync->timed_out ||
          (k > 0 && !wait_counter(&p.sync->done[k - 1], (unsigned)p.total_blocks, &p.sync->timed_out,
                                  kWaitTimeoutNs)))
        tk = -1;
      s_ticket = tk;
    }
    __syncthreads();
    t = s_ticket;
    if (t < 0) return;  // a wait gave up: the host reports it
  }
  const int k = t / p.total_blocks;
  const int w = t - k * p.total_blocks;
  const int ks = p.k0 + k;
  const int q = batch_sim_of(p, w);
  const StepArgs &a = p.v[q][ks % 6];
  const int64_t step = p.t0[q] + ks;
  if (a.parity)
    step_block<ST, LAYOUT, NS, 1, DET, RS, PHYS>(a, w - p.block_start[q], step);
  else
    step_block<ST, LAYOUT, NS, 0, DET, RS, PHYS>(a, w - p.block_start[q], step);
  if (p.n_steps > 1) {
    __syncthreads();  // every thread's writes of this block precede the release
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&p.sync->done[k], 1u);
    }
  }
}

// Per-plane FP64 sums of the current state: one block per plane. Columns:
// rho_C, rho_R, rho_P, rho_P u_z over the plane's fluid cells (u_z the
// carrier's, or the barycentric one when a.bary), and the raw
// wall hits A^R, A^P of the last step over the plane's catalytic nodes.
// Inlet/outlet planes give zeros.
template <int ST, int LAYOUT, int NS, int ODD, bool DET>
__global__ void __launch_bounds__(kBlock) plane_sums_kernel(const ObsArgs o) {
  const StepArgs &a = o.s;
  const int z = blockIdx.x;
  const int64_t plane = (int64_t)a.nx * a.ny;
  const bool bc = !a.periodic_z && (z == 0 || z == a.nz - 1);
  double s[kPlaneCols] = {0, 0, 0, 0, 0, 0};
  if (!bc) {
    const int64_t lo = o.lat_plane[z], hi = o.lat_plane[z + 1];
    for (int64_t Lw = lo + threadIdx.x; Lw < hi; Lw += kBlock) {
      const int32_t L = (int32_t)Lw;
      const int32_t cell = (LAYOUT == LBM_LAYOUT_DENSE) ? L : a.fcell[L];
      if (LAYOUT == LBM_LAYOUT_DENSE && a.mask[cell]) continue;
      const int32_t xy = cell - z * (int32_t)plane;
      const int y = xy / a.nx;
      const int x = xy - y * a.nx;
      const Nbr nb(cell, x, y, z, a.nx, a.ny, a.nz, a.periodic_z);
      float f[NS][kQ];
      load_cell<ST, LAYOUT, NS, ODD, DET>(a, L, nb, a.nbm[L], f);
      float drho = 0.f, jz = 0.f, rR = 0.f, rP = 0.f, jzs = 0.f;
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        drho += f[0][i];
        jz += cz(i) * f[0][i];
        if (NS > 1) rR += f[1][i];
        if (NS > 2) rP += f[NS - 1][i];
#pragma unroll
        for (int sp = 1; sp < NS; ++sp) jzs += cz(i) * f[sp][i];
      }
      s[0] += 1.0 + (double)drho;
      s[1] += rR;
      s[2] += rP;
      const float uz = a.bary ? (jz + jzs) / ((1.0f + drho) + (rR + rP)) : jz / (1.0f + drho) + 0.5f * a.g_z;
      s[3] += (double)rP * (double)uz;
    }
    if (NS > 1) {
      for (int64_t k = o.node_plane[z] + threadIdx.x; k < o.node_plane[z + 1]; k += kBlock) {
        s[4] += hits_d<DET>(a, 0, k);
        if (NS > 2) s[5] += hits_d<DET>(a, 1, k);
      }
    }
  }
  // block reduction in FP64, fixed order
  __shared__ double sh[kPlaneCols][kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kPlaneCols; ++k) {
    double v = warp_sum_d(s[k]);
    if (lane == 0) sh[k][wid] = v;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < kPlaneCols; ++k) {
      double v = (lane < kBlock / 32) ? sh[k][lane] : 0.0;
      v = warp_sum_d(v);
      if (lane == 0) o.plane_sums[kPlaneCols * (int64_t)z + k] = v;
    }
  }
}

// Dense export of a field (which >= 0) or of all populations (which < 0).
template <int ST, int LAYOUT, int NS, int ODD, bool DET>
__global__ void __launch_bounds__(kBlock) export_kernel(const StepArgs a, int which, float *dst, int64_t n) {
  const int64_t Lw = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (Lw >= a.n_lat) return;
  const int32_t L = (int32_t)Lw;
  const int32_t plane = a.nx * a.ny;
  const int32_t cell = (LAYOUT == LBM_LAYOUT_DENSE) ? L : a.fcell[L];
  if (LAYOUT == LBM_LAYOUT_DENSE && a.mask[cell]) return;
  const int z = cell / plane;
  // inlet/outlet planes hold no state of their own (their upwind cells lie
  // outside the box): leave them at 0
  if (!a.periodic_z && (z == 0 || z == a.nz - 1)) return;
  const int32_t xy = cell - z * plane;
  const int y = xy / a.nx;
  const int x = xy - y * a.nx;
  const Nbr nb(cell, x, y, z, a.nx, a.ny, a.nz, a.periodic_z);
  float f[NS][kQ];
  load_cell<ST, LAYOUT, NS, ODD, DET>(a, L, nb, a.nbm[L], f);
  if (which < 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < kQ; ++i) dst[(int64_t)(s * kQ + i) * n + cell] = f[s][i];
    return;
  }
  // velocity: the carrier's, or the barycentric one over every array
  float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, rs[3] = {0.f, 0.f, 0.f}, js[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    drho += f[0][i];
    jx += cx(i) * f[0][i];
    jy += cy(i) * f[0][i];
    jz += cz(i) * f[0][i];
#pragma unroll
    for (int s = 1; s < NS; ++s) {
      rs[s] += f[s][i];
      js[0] += cx(i) * f[s][i];
      js[1] += cy(i) * f[s][i];
      js[2] += cz(i) * f[s][i];
    }
  }
  const float rho = 1.0f + drho;
  const float rho_u = a.bary ? rho + (rs[1] + rs[2]) : rho;
  if (a.bary) {
    jx += js[0];
    jy += js[1];
    jz += js[2];
  }
  float v = 0.f;
  switch (which) {
    case LBM_FIELD_RHO_C: v = rho; break;
    case LBM_FIELD_DRHO_C: v = drho; break;
    case LBM_FIELD_RHO_R: v = rs[1]; break;
    case LBM_FIELD_RHO_P: v = rs[2]; break;
    case LBM_FIELD_UX: v = jx / rho_u; break;
    case LBM_FIELD_UY: v = jy / rho_u; break;
    case LBM_FIELD_UZ: v = a.bary ? jz / rho_u : jz / rho_u + 0.5f * a.g_z; break;
    default: break;
  }
  dst[cell] = v;
}

#define LBM_DISPATCH_ONE(LYV, NSV, ODDV, DETV, ...) \
  do {                                              \
    constexpr int LY = LYV;                         \
    constexpr int NSC = NSV;                        \
    constexpr int OD = ODDV;                        \
    constexpr bool DT = DETV;                       \
    (void)LY; (void)NSC; (void)OD; (void)DT;        \
    __VA_ARGS__;                                    \
  } while (0)
#define LBM_DISPATCH_D(LYV, NSV, ODDV, DET_, ...)                                            \
  do {                                                                                     \
    if (DET_) LBM_DISPATCH_ONE(LYV, NSV, ODDV, true, __VA_ARGS__);                         \
    else LBM_DISPATCH_ONE(LYV, NSV, ODDV, false, __VA_ARGS__);                             \
  } while (0)
#define LBM_DISPATCH_O(LYV, NSV, ODD_, DET_, ...)                                            \
  do {                                                                                     \
    if (ODD_) LBM_DISPATCH_D(LYV, NSV, 1, DET_, __VA_ARGS__);                              \
    else LBM_DISPATCH_D(LYV, NSV, 0, DET_, __VA_ARGS__);                                   \
  } while (0)
#define LBM_DISPATCH_N(LYV, NS_, ODD_, DET_, ...)                                            \
  do {                                                                                     \
    if ((NS_) == 2) LBM_DISPATCH_O(LYV, 2, ODD_, DET_, __VA_ARGS__);                       \
    else LBM_DISPATCH_O(LYV, 3, ODD_, DET_, __VA_ARGS__);                                  \
  } while (0)
// layout x species x parity x deterministic accumulation
#define LBM_DISPATCH_LNS(LAYOUT_, NS_, ODD_, DET_, ...)                                      \
  do {                                                                                     \
    if ((LAYOUT_) == LBM_LAYOUT_DENSE) LBM_DISPATCH_N(LBM_LAYOUT_DENSE, NS_, ODD_, DET_, __VA_ARGS__); \
    else LBM_DISPATCH_N(LBM_LAYOUT_FLUID, NS_, ODD_, DET_, __VA_ARGS__);                   \
  } while (0)

// RS (the random sputtering matrix) and PHYS (carrier velocity; barycentric
// velocity; validation channel: inert solid, body force, species relaxation
// time) are compile-time parameters, so that the default kernels carry none
// of the other modes' code.
template <int ST, bool RS, int PHYS>
cudaError_t launch_step_st(const StepArgs &a, int layout, int ns, int parity, cudaStream_t st) {
  const int64_t work = a.n_lat > a.n_nodes ? a.n_lat : a.n_nodes;
  const unsigned grid = (unsigned)((work + kBlock - 1) / kBlock);
  if (grid == 0) return cudaSuccess;
  LBM_DISPATCH_LNS(layout, ns, parity, a.det, step_kernel<ST, LY, NSC, OD, DT, RS, PHYS><<<grid, kBlock, 0, st>>>(a));
  return cudaGetLastError();
}

template <int ST, bool RS, int PHYS>
cudaError_t launch_batch_st(const BatchLaunch &p, int layout, int ns, int det, cudaStream_t st) {
  if (p.total_blocks <= 0 || p.n_sims <= 0 || p.n_steps <= 0) return cudaSuccess;
  if (p.n_steps > 1 && !p.sync) return cudaErrorInvalidValue;
  if ((int64_t)p.n_steps * p.total_blocks >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)(p.n_steps * p.total_blocks);
  LBM_DISPATCH_LNS(layout, ns, 0, det, batch_step_kernel<ST, LY, NSC, DT, RS, PHYS><<<grid, kBlock, 0, st>>>(p));
  return cudaGetLastError();
}

template <int ST>
cudaError_t launch_plane_sums_st(const ObsArgs &o, int layout, int ns, cudaStream_t st) {
  LBM_DISPATCH_LNS(layout, ns, o.parity, o.s.det, plane_sums_kernel<ST, LY, NSC, OD, DT><<<o.s.nz, kBlock, 0, st>>>(o));
  return cudaGetLastError();
}

template <int ST>
cudaError_t launch_export_st(const StepArgs &a, int parity, int layout, int ns, int which, float *dst,
                             cudaStream_t st) {
  const unsigned grid = (unsigned)((a.n_lat + kBlock - 1) / kBlock);
  if (grid == 0) return cudaSuccess;
  const int64_t n = (int64_t)a.nx * a.ny * a.nz;
  LBM_DISPATCH_LNS(layout, ns, parity, a.det,
                   export_kernel<ST, LY, NSC, OD, DT><<<grid, kBlock, 0, st>>>(a, which, dst, n));
  return cudaGetLastError();
}

#define LBM_INSTANTIATE_STEP(ST, RS, PHYS)                                                           \
  template cudaError_t launch_step_st<ST, RS, PHYS>(const StepArgs &, int, int, int, cudaStream_t);   \
  template cudaError_t launch_batch_st<ST, RS, PHYS>(const BatchLaunch &, int, int, int, cudaStream_t);
#define LBM_INSTANTIATE_STORAGE(ST)                                                                    \
  LBM_INSTANTIATE_STEP(ST, false, kPhysCarrier)                                                               \
  template cudaError_t launch_plane_sums_st<ST>(const ObsArgs &, int, int, cudaStream_t);             \
  template cudaError_t launch_export_st<ST>(const StepArgs &, int, int, int, int, float *, cudaStream_t);

}  // namespace lbm
