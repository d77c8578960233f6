// Fused collide-stream-boundary kernel and state readers, templated on the
// population storage. Included once per storage type and variant
// (step_f32.cu, step_f16.cu, step_bf16.cu, ...) so the units compile in
// parallel.
//
// Time stepping follows the lattice BGK equation of the paper's Appendix
// (Eq. LBE, Eq. feq, one omega for every species), with species relaxed
// towards an equilibrium built on the carrier velocity, halfway bounce-back
// of the carrier at solid links, and the sputtering law (Appendix,
// Eq. f_P_in) with S_ij = 1/b(x) at catalytic nodes.
//
// Streaming is in place (AA pattern): one population array per kind. Each
// cell owns 19 pointer slots per array, P_k, and a step loads the 19 values
// behind them and stores 19 new values to the same places:
//   - even step: P_k = own slot k. The load is the incoming population of
//     direction k; the store is the outgoing f*_opp(k) (so f*_i lands in own
//     slot opp(i));
//   - odd step: P_k = slot k of the neighbour x + c_k. The load is the
//     incoming population of direction opp(k) (the neighbour's even-step
//     output f*_opp(k)(x - c_opp(k))); the store is the outgoing f*_k, which
//     the neighbour reads as its incoming k after the step. After an odd
//     step the arrays hold the streamed populations in natural order again.
//   - when x + c_k is solid (or, on an inlet/outlet plane, outside the box)
//     the odd step's P_k is the cell's own slot opp(k): the store of f*_k
//     there is the halfway bounce-back that the next step reads as incoming
//     opp(k); the even step's own-slot pointers give the same by
//     construction.
//   - species arriving from a catalytic solid are rebuilt from that node's
//     wall hits of the previous step (A_prev) by the sputtering law; species
//     leaving towards one are added to the node's hits of this step (A_cur).
//     So the wall re-emits one step after the hit, the timing of bounce-back,
//     with no grid-wide synchronisation. A 3-deep ring (prev, cur, next) lets
//     every step clear the buffer of the step after.
//   - inlet plane z=0 / outlet plane z=nz-1: equilibrium with the velocity of
//     plane 1 / nz-2 from the previous step (and, at the outlet, the species
//     densities of plane nz-2), passed through a double-buffered plane cache.
//
// All arithmetic is on the stored scaled deviations d_i = (f_i - w_i rho_ref)
// / w_i (rho_ref = 1 for the carrier, 0 for the species): drho = sum w d,
// j = sum w c d (the w_i rho_ref parts cancel since sum w c = 0),
// rho = rho_ref + drho, u = j / rho. With P_i = 3 c.u + 4.5 (c.u)^2 - 1.5 u^2,
// the same for every array that relaxes towards the same u, the equilibria
// are deq_i = drho + rho P_i (carrier) and rho_s + rho_s P_i (species), and
// d*_i = (1 - omega) d_i + omega deq_i. The reactant and product of a slot
// move as one pair and relax with packed FP32x2 arithmetic.
#pragma once

#include <algorithm>

#include "lbm_internal.h"

namespace lbm {

// Population layout: two warp-blocked arrays (carrier a.f, species a.fs).
// Entry e, slot k lives at element (e / 32) 608 + 32 k + e % 32 of each
// (608 = 19 x 32): a warp's 32 consecutive entries are contiguous for every
// slot, and all slots of an entry are compile-time offsets from one base.
__device__ __forceinline__ int64_t ent_off(int32_t e) { return (int64_t)(e >> 5) * (kQ * 32) + (e & 31); }
// ent_off modulo 2^32: the difference of two of these is the exact element
// distance between two entries whenever that distance is below 2^31
__device__ __forceinline__ uint32_t ent_off32(int32_t e) { return (uint32_t)e + ((uint32_t)e >> 5) * (uint32_t)(kQ * 32 - 32); }

// slots whose neighbour lies below / above the cell in z
constexpr uint32_t kDownBits = (1u << 6) | (1u << 12) | (1u << 13) | (1u << 16) | (1u << 17);
constexpr uint32_t kUpBits = (1u << 5) | (1u << 11) | (1u << 14) | (1u << 15) | (1u << 18);

// Population loads name their cache operator (ld.global.ca): never the
// non-coherent read-only path, which a const __restrict__ pointer would
// allow. Within one multi-step batched launch a CTA reads populations that
// other CTAs wrote earlier in the same launch; ordinary loads observe them
// after the step-ordering acquire, non-coherent loads need not.
// Population stores are streaming stores (st.global.cs): each stored value
// is read once, by the next step; coherence is unchanged.
template <typename T>
__device__ __forceinline__ T ld_pop(const T *p) {
  return __ldca(p);
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

// Species (R, P) re-emitted by the catalytic node `node` along its outgoing
// link i (the incoming population of direction i of the fluid cell behind
// it), in the units of the stored species (scaled deviations d = f / w).
template <int ST, int NS, bool DET>
__device__ __forceinline__ float2 emission(bool rs, const StepArgs &a, int i, int32_t node, int32_t node_cell) {
  const float ib = __fmul_rn(emit_scale(rs, a, node), inv_wq(i) * Pop<ST, NS>::kSp);
  const int64_t e = emit_index(rs, a, i, node, node_cell);
  const float AR = acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, e, LBM_NACC(a)));
  float2 v;
  v.x = __fmul_rn(__fmul_rn(a.em_R, AR), ib);
  v.y = 0.0f;
  if (NS > 2) {
    const float AP = acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, a.acc_row + e, LBM_NACC(a)));
    v.y = __fmul_rn(fmaf(a.em_PR, AR, __fmul_rn(a.em_P, AP)), ib);
  }
  return v;
}

// Populations of lattice entry L at the current time as deviations
// g = f - w rho_ref (species unscaled), as a two-lattice scheme would hold
// them (natural order), for a state of parity ODD (ODD = 1: the last
// completed step was an even one). For the observables and exports.
template <int ST, int LAYOUT, int NS, int ODD, bool DET>
__device__ __forceinline__ void load_cell(const StepArgs &a, int32_t L, const Nbr &nb, uint32_t nbm,
                                          float (&f)[NS][kQ]) {
  using P = Pop<ST, NS>;
  const typename P::C *Cb = static_cast<const typename P::C *>(a.f);
  const typename P::S *Sb = static_cast<const typename P::S *>(a.fs);
  const int64_t own = ent_off(L);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const bool solid_up = (i != 0) && ((nbm >> opp(i)) & 1u);
    int64_t base = own;
    int slot = i;
    if (ODD && i != 0 && !solid_up) {
      const int32_t src = nb.at(-cx(i), -cy(i), -cz(i));
      base = ent_off(LAYOUT == LBM_LAYOUT_DENSE ? src : __ldg(a.idx + LBM_OFF(a, kChkIdx, 0, src, LBM_NCELLS(a))));
      slot = opp(i);
    }
    // carrier: with a solid upwind, the cell's own reversed post-collision
    // population sits in slot i in both parities
    f[0][i] = wq(i) * P::c_val(ld_pop(Cb + LBM_OFF(a, kChkPop, 0, base + 32 * slot, LBM_NPOP(a))));
    if (NS > 1) {
      float2 s = P::s_val(ld_pop(Sb + LBM_OFF(a, kChkPop, 0, base + 32 * slot, LBM_NPOP(a))));
      if (solid_up) {
        const int32_t node_cell = nb.at(-cx(i), -cy(i), -cz(i));
        const int32_t node = __ldg(a.idx + LBM_OFF(a, kChkIdx, 0, node_cell, LBM_NCELLS(a)));
        // inert solid or species bounce-back: every array's own reversed
        // population, as the carrier's
        if (!(node < 0 || a.sp_bb)) s = emission<ST, NS, DET>(a.rs != 0, a, i, node, node_cell);
      }
      f[1][i] = wq(i) * P::kSpInv * s.x;
      if (NS > 2) f[2][i] = wq(i) * P::kSpInv * s.y;
    }
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// 36 w_i: the lattice weights as exact integer multiples of 1/36
__host__ __device__ constexpr float w36(int i) { return i == 0 ? 12.0f : (i <= 6 ? 2.0f : 1.0f); }
// x / 36 without bias: x h + x l with h = 1/36 rounded to float and
// l = 1/36 - h rounded to float (1/36 to about 48 bits)
__device__ __forceinline__ float div36(float x) {
  constexpr float h = 1.0f / 36.0f;
  constexpr float l = (float)(1.0 / 36.0 - (double)(1.0f / 36.0f));
  return fmaf(x, l, __fmul_rn(x, h));
}
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// This thread's shared-memory slot for the odd step's offset along c_k
// (k = 1 .. 16): the warp's [16][32] slice of a block-wide array (volatile,
// so that the store reads it back instead of keeping a register copy).
// 16 KB per block, 64 KB for four blocks; the last two offsets stay in
// registers. Measured on the 512x512x1024 box, 16-bit odd steps are 1.8%
// faster than with all 18 offsets in shared memory (73.7 KB for four
// blocks), which leaves the SM less L1.
__device__ __forceinline__ volatile int32_t &rel_slot(int k) {
  __shared__ int32_t s_rel[kWarpsPerBlock * 16 * 32];
  return *((volatile int32_t *)s_rel + (threadIdx.x >> 5) * (16 * 32) + (k - 1) * 32 + (threadIdx.x & 31));
}

// Update of one cell: load the 19 slots of both arrays, moments, relaxation
// (or the inlet/outlet equilibrium), store to the same slots. FAST: the
// whole warp lies away from the inlet/outlet and halo planes. Without WALL
// it has no solid neighbour either; with WALL (nbm given) the odd step's
// pointers of its solid links fall back to the cell's own reversed slot.
template <int ST, int LAYOUT, int NS, int ODD, bool DET, bool FAST, bool RS, int PHYS, bool WALL = false,
          bool SMEM = false, bool UNI = false>
__device__ __forceinline__ void cell_update(const StepArgs &a, int32_t L, int32_t cell, uint32_t nbm, int64_t t,
                                            float (&flux)[6]) {
  using P = Pop<ST, NS>;
  using CT = typename P::C;
  using STy = typename P::S;
  const int32_t plane = a.nx * a.ny;
  // cell coordinates and neighbours: not needed on even fast steps (two
  // integer divisions saved)
  int z = 0, y = 0, x = 0;
  int32_t xy = 0;
  Nbr nb;
  if (!FAST || ODD) {
    z = (int)fast_div((uint32_t)cell, a.div_plane_m, a.div_sh & 0xffu, (a.div_sh >> 8) & 0xffu);
    xy = cell - z * plane;
    y = (int)fast_div((uint32_t)xy, a.div_nx_m, (a.div_sh >> 16) & 0xffu, a.div_sh >> 24);
    x = xy - y * a.nx;
    nb = Nbr(cell, x, y, z, a.nx, a.ny, a.nz, a.periodic_z);
  }
  (void)x;
  (void)y;
  // open ends (inlet below, outlet above): not periodic and not a halo
  const bool open_lo = !a.periodic_z && !a.halo_lo, open_hi = !a.periodic_z && !a.halo_hi;
  const bool bc = !FAST && ((open_lo && z == 0) || (open_hi && z == a.nz - 1));
  const int fsel = FAST ? -1
                        : ((open_lo && z == 0)             ? 0
                           : (open_lo && z == 1)          ? 1
                           : (open_hi && z == a.nz - 2)   ? 2
                           : (open_hi && z == a.nz - 1)   ? 3
                                                          : -1);
  // slots whose neighbour is solid or outside the box: the odd step's
  // pointer falls back to the cell's own reversed slot
  const uint32_t solid = (FAST && !WALL) ? 0u : nbm;
  const uint32_t redirect = solid | (bc ? (z == 0 ? kDownBits : kUpBits) : 0u);

  CT *const Co = static_cast<CT *>(a.f) + ent_off(L);
  STy *const So = static_cast<STy *>(a.fs) + ent_off(L);
  const int64_t own = ent_off(L);  // (bounds checks)

  // Odd steps: rel[k], the element offset of slot k's pointer from the
  // entry's own slot k: to the neighbour's entry (fluid-only addressing:
  // idx[cell + c_k]; in a region warp (UNI), whose numbering is the cells'
  // own order, L plus the neighbour's cell offset), or, for a solid or
  // outside neighbour, to the cell's own reversed slot. One 32-bit value per
  // slot; the node number of a solid neighbour is read again from idx where
  // a wall link needs it.
  // Odd fast steps park 16 of the 18 offsets in shared memory (this warp's
  // [16][32] slice) until the store, instead of holding them in registers
  // across the arithmetic: with them the kernel needs 80 registers and
  // spills, without them it fits the 64 of four blocks per SM.
  constexpr bool SREL = ODD && FAST && SMEM;
  int32_t rel[kQ];
  const uint32_t own32 = ent_off32(L);
#pragma unroll
  for (int k = 0; k < kQ; ++k) {
    rel[k] = 0;
    if (ODD && k != 0) {
      if ((!FAST || WALL) && ((redirect >> k) & 1u)) {
        rel[k] = 32 * (opp(k) - k);
      } else {
        const int32_t c2 = nb.at(cx(k), cy(k), cz(k));
        int32_t e;
        if constexpr (LAYOUT == LBM_LAYOUT_DENSE) e = c2;
        else if constexpr (UNI) e = L + (c2 - cell);
        else e = __ldg(a.idx + LBM_OFF(a, kChkIdx, 0, c2, LBM_NCELLS(a)));
        rel[k] = (int32_t)(ent_off32(e) - own32);
      }
      if constexpr (SREL) { if (k <= 16) rel_slot(k) = rel[k]; }
    }
  }
  // ---- load ----
  // The 16-bit formats keep the species as loaded (one 32-bit register per
  // slot) and convert them where they are used, which holds 19 registers
  // fewer than the converted pairs.
  constexpr bool RAW = ST != LBM_FP32;
  float cv[kQ];
  float2 sv[kQ];
  STy sraw[kQ];
  if (!bc) {
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
      const int i = ODD ? opp(k) : k;  // the incoming direction this slot holds
      cv[i] = P::c_val(ld_pop(Co + LBM_OFF(a, kChkPop, own, rel[k] + 32 * k, LBM_NPOP(a))));
      if (NS > 1) {
        sraw[i] = ld_pop(So + LBM_OFF(a, kChkPop, own, rel[k] + 32 * k, LBM_NPOP(a)));
        if (!RAW) sv[i] = P::s_val(sraw[i]);
      } else {
        sraw[i] = STy{};
        sv[i] = f2(0.0f);
      }
    }
    // (species arriving from a catalytic node: node_emit_kernel has written
    // the sputtering law's value into the slot, the cell's own slot i)
  } else {
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      cv[i] = 0.0f;
      sv[i] = f2(0.0f);
      sraw[i] = STy{};
    }
  }
  // species pair of incoming direction i; `again`: convert afresh (the empty
  // asm keeps the compiler from holding the first conversion instead)
  auto spc = [&](int i, bool again) -> float2 {
    if constexpr (!RAW || NS < 2) {
      return sv[i];
    } else {
      STy r = sraw[i];
      if (again) {
        if constexpr (sizeof(STy) == 2) asm volatile("" : "+h"(r));
        else asm volatile("" : "+r"(r));
      }
      return P::s_val(r);
    }
  };

  // ---- moments ----
  constexpr bool BARY = PHYS == kPhysBary;
  float drho, ux, uy, uz;
  float2 rs;  // species densities (stored units)
  if (!bc) {
    // Moments. 16-bit storage: sums with the exact integer weights
    // 36 w_i = 12, 2, 1 and one division by 36 at the end, formed as
    // x h + x l with h + l = 1/36 to twice float precision so that its
    // rounding has no bias (float weights 1/3, 1/18, 1/36 sum to 1 + 1.4e-8
    // and would scale every collision's mass by that factor). FP32 storage:
    // see below.
    float j36x = 0.f, j36y = 0.f, j36z = 0.f, d36, inv36;
    float2 rs36, js[3] = {f2(0.f), f2(0.f), f2(0.f)};
    if constexpr (ST == LBM_FP32) {
      // FP32 storage: weighted sums population by population, w d rounded
      // once and added, as j = sum w c d and rho = sum w d (the float
      // weights carry a common relative excess of ~1e-8, which here scales
      // j and rho alike). Kept because it is the form whose fixed points lie
      // closest to the FP64 solution in long steady flows, where every
      // rounding repeats identically at every step.
      d36 = 0.f;
      rs36 = f2(0.f);
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const float wd = __fmul_rn(wq(i), cv[i]);
        d36 = __fadd_rn(d36, wd);
        if (cx(i)) j36x = __fadd_rn(j36x, cx(i) * wd);
        if (cy(i)) j36y = __fadd_rn(j36y, cy(i) * wd);
        if (cz(i)) j36z = __fadd_rn(j36z, cz(i) * wd);
        if (NS > 1) {
          rs36 = fma2(f2(wq(i)), sv[i], rs36);
          if (BARY) {
            if (cx(i)) js[0] = fma2(f2(cx(i) * wq(i)), sv[i], js[0]);
            if (cy(i)) js[1] = fma2(f2(cy(i) * wq(i)), sv[i], js[1]);
            if (cz(i)) js[2] = fma2(f2(cz(i) * wq(i)), sv[i], js[2]);
          }
        }
      }
    } else {
      // 16-bit storage: sums and differences of opposite slots
      float sa = 0.f, sd = 0.f;
      float2 rsa = f2(0.f), rsd = f2(0.f);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const int i = 2 * q + 1;
        const float s = __fadd_rn(cv[i], cv[i + 1]), dd = __fsub_rn(cv[i], cv[i + 1]);
        if (i <= 6) sa = __fadd_rn(sa, s); else sd = __fadd_rn(sd, s);
        const float w = w36(i);
        if (cx(i)) j36x = fmaf((float)cx(i) * w, dd, j36x);
        if (cy(i)) j36y = fmaf((float)cy(i) * w, dd, j36y);
        if (cz(i)) j36z = fmaf((float)cz(i) * w, dd, j36z);
        if (NS > 1) {
          const float2 s2 = add2(spc(i, false), spc(i + 1, false));
          if (i <= 6) rsa = add2(rsa, s2); else rsd = add2(rsd, s2);
          if (BARY) {
            const float2 d2 = fma2(f2(-1.0f), spc(i + 1, false), spc(i, false));
            if (cx(i)) js[0] = fma2(f2(cx(i) * w), d2, js[0]);
            if (cy(i)) js[1] = fma2(f2(cy(i) * w), d2, js[1]);
            if (cz(i)) js[2] = fma2(f2(cz(i) * w), d2, js[2]);
          }
        }
      }
      d36 = fmaf(12.0f, cv[0], fmaf(2.0f, sa, sd));
      rs36 = fma2(f2(12.0f), spc(0, false), fma2(f2(2.0f), rsa, rsd));
    }
    if constexpr (ST == LBM_FP32) {
      drho = d36;  // (FP32: the sums above are already weighted)
      rs = rs36;
    } else {
      drho = div36(d36);
      rs = make_float2(div36(rs36.x), div36(rs36.y));
    }
    // (FP32 sums are already divided by 36: the velocity divides by rho,
    // the 16-bit ones by 36 rho)
    constexpr float kR = (ST == LBM_FP32) ? 1.0f : 36.0f;
    if (BARY) {
      // u = (j_C + j_R + j_P) / (rho_C + rho_R + rho_P)
      const float msp = __fmul_rn(__fadd_rn(rs.x, rs.y), P::kSpInv);
      inv36 = 1.0f / __fmul_rn(kR, __fadd_rn(__fadd_rn(1.0f, drho), msp));
      j36x = fmaf(__fadd_rn(js[0].x, js[0].y), P::kSpInv, j36x);
      j36y = fmaf(__fadd_rn(js[1].x, js[1].y), P::kSpInv, j36y);
      j36z = fmaf(__fadd_rn(js[2].x, js[2].y), P::kSpInv, j36z);
    } else {
      inv36 = (ST == LBM_FP32) ? 1.0f / __fadd_rn(1.0f, drho) : 1.0f / fmaf(36.0f, drho, 36.0f);
    }
    const float inv_rho = inv36, jx = j36x, jy = j36y, jz = j36z;
    ux = __fmul_rn(jx, inv_rho);
    uy = __fmul_rn(jy, inv_rho);
    uz = __fmul_rn(jz, inv_rho);
    if (PHYS == kPhysChannel) uz = fmaf(0.5f, a.g_z, uz);  // body force: the velocity half a step on
    if (!FAST && ((open_lo && z == 1) || (open_hi && z == a.nz - 2))) {
      // plane cache: u_x, u_y, u_z, rho_R, rho_P at ub[0], ub[plane], ... (the check bounds the last)
      float *ub = a.ub_cur + LBM_OFF(a, kChkUb, 0, (int64_t)(z == 1 ? 0 : 5) * plane + xy,
                                     LBM_NUB(a) - 4 * (int64_t)plane);
      ub[0] = ux;
      ub[plane] = uy;
      ub[2 * (int64_t)plane] = uz;
      if (NS > 1) ub[3 * (int64_t)plane] = rs.x * P::kSpInv;
      if (NS > 2) ub[4 * (int64_t)plane] = rs.y * P::kSpInv;
    }
  } else {
    const float *ub = a.ub_prev + LBM_OFF(a, kChkUb, 0, (int64_t)(z == 0 ? 0 : 5) * plane + xy,
                                          LBM_NUB(a) - 4 * (int64_t)plane);
    ux = ub[0];
    uy = ub[plane];
    uz = ub[2 * (int64_t)plane];
    if (z == 0 && a.vel_in) {  // velocity inlet: (0, 0, u_in)
      ux = 0.f;
      uy = 0.f;
      uz = a.u_in;
    }
    drho = (z == 0) ? a.drho_in : a.drho_out;
    rs = (z == 0) ? make_float2(a.c_in * P::kSp, 0.0f)
                  : make_float2(ub[3 * (int64_t)plane] * P::kSp, NS > 2 ? ub[4 * (int64_t)plane] * P::kSp : 0.0f);
  }

  // ---- relaxation (or equilibrium on the inlet/outlet planes) and store ----
  // (every multiply-add below is written out, as an FMA or as a rounded
  // multiply and add, so that each kernel that inlines this function - the
  // fast, general and batched ones - computes bit-identical results)
  const float rho = __fadd_rn(1.0f, drho);
  const float om = bc ? 1.0f : a.omega;
  const float om_s = bc ? 1.0f : (PHYS == kPhysCarrier ? a.omega : a.omega_s);
  const float wr = __fmul_rn(om, rho), wd = __fmul_rn(om, drho), omc = __fsub_rn(1.0f, om);
  const float2 wrs = __fmul2_rn(f2(om_s), rs), omc_s = f2(__fsub_rn(1.0f, om_s));
  const float Ux = __fmul_rn(3.0f, ux), Uy = __fmul_rn(3.0f, uy), Uz = __fmul_rn(3.0f, uz);
  const float u2 = __fmul_rn(1.5f, fmaf(uz, uz, fmaf(uy, uy, __fmul_rn(ux, ux))));
  const float fz = (PHYS == kPhysChannel && !bc) ? __fmul_rn(__fmul_rn(fmaf(-0.5f, a.omega, 1.0f), rho), a.g_z) : 0.0f;
  const uint32_t h = (ST == LBM_FP32) ? 0u : mix32(((uint32_t)L + a.hash_base) ^ step_seed_of(t, a.seed_mix));
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    // P_i from the pair (i, opp(i)): q = 4.5 (c.u)^2 - 1.5 u^2 shared, +-3 c.u
    const int ip = (i == 0) ? 0 : ((i & 1) ? i : i - 1);
    float cu, Pi;
    if constexpr (ST == LBM_FP32) {
      // per direction: 3 c.u from the velocity components, then
      // (3 c.u + 4.5 (c.u)^2) - 1.5 u^2
      const float cd = __fmul_rn(3.0f, __fadd_rn(__fadd_rn(cx(ip) * ux, cy(ip) * uy), cz(ip) * uz));
      const float ci = (i & 1) || i == 0 ? cd : -cd;
      cu = cd;
      Pi = __fsub_rn(fmaf(__fmul_rn(0.5f, ci), ci, ci), u2);
    } else {
      cu = __fadd_rn(__fadd_rn(cx(ip) * Ux, cy(ip) * Uy), cz(ip) * Uz);
      const float qq = fmaf(__fmul_rn(0.5f, cu), cu, -u2);
      Pi = (i == 0) ? -u2 : ((i & 1) ? __fadd_rn(qq, cu) : __fsub_rn(qq, cu));
    }
    // FP32 storage keeps d + omega (deq - d), whose rounding shrinks with
    // the distance from equilibrium; the 16-bit formats, whose storage
    // rounding is far coarser, take (1 - omega) d + omega deq (two FMAs)
    float c_out;
    if constexpr (ST == LBM_FP32) c_out = fmaf(om, __fsub_rn(fmaf(rho, Pi, drho), cv[i]), cv[i]);
    else c_out = fmaf(wr, Pi, fmaf(omc, cv[i], wd));
    if (PHYS == kPhysChannel && !bc && a.g_z != 0.f) {
      // body force F = rho g along z, Guo, Zheng and Shi (2002): in scaled
      // deviations the source adds (1 - omega/2) [3 (c_iz - u_z) + 9 (c_i . u) c_iz] F_z
      const float cui = (i & 1) || i == 0 ? cu : -cu;
      c_out = fmaf(fz, fmaf(cui, 3.0f * cz(i), __fmul_rn(3.0f, __fsub_rn((float)cz(i), uz))), c_out);
    }
    float2 s_out;
    if constexpr (ST == LBM_FP32) s_out = fma2(f2(om_s), fma2(f2(-1.0f), sv[i], fma2(f2(Pi), rs, rs)), sv[i]);
    else s_out = fma2(omc_s, spc(i, true), fma2(f2(Pi), wrs, wrs));
    const int k = ODD ? i : opp(i);  // the slot that receives f*_i
    // (odd steps: the offset passes through an empty asm so that the store
    // address is formed again from the 32-bit offset, instead of the 64-bit
    // load addresses of all 19 slots being held across the arithmetic)
    int32_t rk = rel[k];
    if constexpr (SREL) {
      if (k != 0 && k <= 16) rk = rel_slot(k);
      else if (k != 0) asm volatile("" : "+r"(rk));
    } else if (ODD) {
      asm volatile("" : "+r"(rk));
    }
    const CT qc = P::c_cv(c_out, h * sr_mul(0, i));
    __stcs(Co + LBM_OFF(a, kChkPop, own, rk + 32 * k, LBM_NPOP(a)), qc);
    STy qs{};
    if (NS > 1) {
      qs = P::s_cv(s_out, h * sr_mul(1, i));
      __stcs(So + LBM_OFF(a, kChkPop, own, rk + 32 * k, LBM_NPOP(a)), qs);
    }
    if (!FAST && i != 0) {
      // inlet / outlet face flows of the stored (rounded) values
      if (fsel >= 0 && !((redirect >> i) & 1u)) {
        const bool up = cz(i) > 0, dn = cz(i) < 0;
        const float sgn =
            ((fsel == 0 || fsel == 2) && up) ? 1.f : (((fsel == 1 || fsel == 3) && dn) ? -1.f : 0.f);
        if (sgn != 0.f) {
          const int o = fsel <= 1 ? 0 : 3;
          const float sw = sgn * wq(i);
          flux[o] = fmaf(sw, P::c_val(qc), flux[o]);
          if (NS > 1) {
            const float2 sq = P::s_val(qs);
            flux[o + 1] = fmaf(sw * P::kSpInv, sq.x, flux[o + 1]);
            if (NS > 2) flux[o + 2] = fmaf(sw * P::kSpInv, sq.y, flux[o + 2]);
          }
        }
      }
      // (species sent towards a catalytic node stay in the redirected slot,
      // where node_hits_kernel sums them)
    }
  }
}

// Face-flow slot of lattice warp W (the warps overlapping planes 0, 1 and
// nz-2, nz-1), or -1.
__device__ __forceinline__ int32_t flux_slot(const StepArgs &a, int32_t W) {
  if (a.periodic_z) return -1;
  if (W < a.n_lo_warps) return W;
  if (W >= a.hi_warp && W < a.n_lat_warps) return a.n_lo_warps + (W - a.hi_warp);
  return -1;
}

// Adds the warp's face flows, summed in FP64 in a fixed order, to its slot.
// Every lane of the warp must call it.
__device__ __forceinline__ void bank_flux(const StepArgs &a, int32_t W, const float (&flux)[6]) {
  const int32_t slot = flux_slot(a, W);
  if (slot < 0) return;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double v = warp_sum_d((double)flux[k]);
    if ((threadIdx.x & 31) == 0) a.flux_cum[6 * (int64_t)slot + k] += v;
  }
}

// ---- Catalytic nodes: the sputtering law (Appendix, Eq. f_P_in) ----
//
// A wall link of node n along c_j joins it to the fluid cell x = n + c_j. In
// both parities of the in-place streaming, x stores the population it sends
// towards n in its own slot j (the halfway bounce-back of the carrier), and
// it reads from that same slot the population that arrives from n along c_j.
// So the species part of the boundary acts on those slots alone, one thread
// per node, around the cell updates of a step:
//   node_emit, before them: bank the previous step's hits of the node, and
//     write into each link's slot what the sputtering law returns along the
//     link (emission);
//   node_hits, after them: the species that reached the node in this step,
//     w_j times each link's stored value, summed over the node's links in a
//     fixed order (or in 64-bit fixed point), into the step's accumulator
//     (under the random matrix, each into the slot of the link it leaves by).
// The carrier's slot keeps its bounce-back. Inert solid is never a node, and
// under species bounce-back (sp_bb) neither kernel runs, so the species
// bounce back too.

// Lattice entries of the fluid cells across the links of the node in cell
// nc (active links in `links`), or -1 where there is no link or the cell is
// in a halo plane (stepped by the neighbouring sub-domain). Every active link
// ends inside the box. All 18 index loads are issued together.
template <int LAYOUT>
__device__ __forceinline__ void link_entries(const StepArgs &a, int32_t nc, uint32_t links, int32_t (&Ls)[kQ]) {
  const int32_t plane = a.nx * a.ny;
  const int z = nc / plane;
  const int32_t xy = nc - z * plane;
  const int y = xy / a.nx;
  const Nbr nb(nc, xy - y * a.nx, y, z, a.nx, a.ny, a.nz, a.periodic_z);
  Ls[0] = -1;
#pragma unroll
  for (int j = 1; j < kQ; ++j) {
    Ls[j] = -1;
    if (((links >> j) & 1u) && !halo_plane(a, z + cz(j))) {
      const int32_t c = nb.at(cx(j), cy(j), cz(j));
      Ls[j] = LAYOUT == LBM_LAYOUT_DENSE ? c : __ldg(a.idx + LBM_OFF(a, kChkIdx, 0, c, LBM_NCELLS(a)));
    }
  }
}

// Emission of node n for step t, and the banking of its previous hits into
// hv (R, P). (t is passed apart from a.t: a batched launch reuses argument
// sets six steps apart.)
template <int ST, int LAYOUT, int NS, bool DET, bool RS>
__device__ __forceinline__ void node_emit(const StepArgs &a, int64_t n, int64_t t, float (&hv)[2]) {
  using P = Pop<ST, NS>;
  using STy = typename P::S;
  hv[0] = hv[1] = 0.f;
  const int32_t nc = __ldg(a.node_cell + LBM_OFF(a, kChkNode, 0, n, a.n_nodes));
  const uint32_t links = __ldg(a.cell_bits + LBM_OFF(a, kChkIdx, 0, nc, LBM_NCELLS(a)));
  int32_t Ls[kQ];
  link_entries<LAYOUT>(a, nc, links, Ls);
  if (RS) {
    for (int32_t k = __ldg(a.node_off + LBM_OFF(a, kChkNode, 0, n, a.n_nodes + 1));
         k < __ldg(a.node_off + LBM_OFF(a, kChkNode, 0, n + 1, a.n_nodes + 1)); ++k) {
      hv[0] += acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, k, LBM_NACC(a)));
      if (NS > 2) hv[1] += acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, a.acc_row + k, LBM_NACC(a)));
    }
  } else {
    hv[0] = acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, n, LBM_NACC(a)));
    if (NS > 2) hv[1] = acc_get<DET>(a.A_prev, LBM_OFF(a, kChkAcc, 0, a.acc_row + n, LBM_NACC(a)));
  }
  STy *const S = static_cast<STy *>(a.fs);
  const uint32_t sd = step_seed_of(t, a.seed_mix);
#pragma unroll
  for (int j = 1; j < kQ; ++j) {
    if (Ls[j] < 0) continue;
    const float2 v = emission<ST, NS, DET>(RS, a, j, (int32_t)n, nc);
    const uint32_t h = (ST == LBM_FP32) ? 0u : mix32(((uint32_t)Ls[j] + a.hash_base) ^ sd);
    S[LBM_OFF(a, kChkPop, 0, ent_off(Ls[j]) + 32 * j, LBM_NPOP(a))] = P::s_cv(v, h * sr_mul(2, j));
  }
}

// Wall hits of node n in step t: the species its links' cells sent towards
// it, into a.A_cur.
template <int ST, int LAYOUT, int NS, bool DET, bool RS>
__device__ __forceinline__ void node_hits(const StepArgs &a, int64_t n, int64_t t) {
  using P = Pop<ST, NS>;
  using STy = typename P::S;
  const int32_t nc = __ldg(a.node_cell + LBM_OFF(a, kChkNode, 0, n, a.n_nodes));
  const uint32_t links = __ldg(a.cell_bits + LBM_OFF(a, kChkIdx, 0, nc, LBM_NCELLS(a)));
  int32_t Ls[kQ];
  link_entries<LAYOUT>(a, nc, links, Ls);
  const STy *const S = static_cast<const STy *>(a.fs);
  STy raw[kQ];
#pragma unroll
  for (int j = 1; j < kQ; ++j)
    raw[j] = Ls[j] >= 0 ? S[LBM_OFF(a, kChkPop, 0, ent_off(Ls[j]) + 32 * j, LBM_NPOP(a))] : STy{};
  int32_t o = 0, m = 0;
  if (RS) {
    o = __ldg(a.node_off + LBM_OFF(a, kChkNode, 0, n, a.n_nodes + 1));
    m = __ldg(a.node_off + LBM_OFF(a, kChkNode, 0, n + 1, a.n_nodes + 1)) - o;
    for (int32_t k = 0; k < m; ++k) {
      acc_clear<DET>(a.A_cur, LBM_OFF(a, kChkAcc, 0, o + k, LBM_NACC(a)));
      if (NS > 2) acc_clear<DET>(a.A_cur, LBM_OFF(a, kChkAcc, 0, a.acc_row + o + k, LBM_NACC(a)));
    }
  }
  acc_t iR = 0ull, iP = 0ull;  // fixed-point sums (DET)
  float fR = 0.f, fP = 0.f;    // FP32 sums, in link order
#pragma unroll
  for (int j = 1; j < kQ; ++j) {
    if (Ls[j] < 0) continue;
    const float2 s = P::s_val(raw[j]);
    // (the population that arrived moves along c_opp(j); w_opp(j) = w_j)
    const float vR = __fmul_rn(wq(j) * P::kSpInv, s.x), vP = __fmul_rn(wq(j) * P::kSpInv, s.y);
    if (RS) {
      const int64_t k = o + rs_rank(a.rs_key, nc, opp(j), t, m);
      acc_put<DET>(a.A_cur, LBM_OFF(a, kChkAcc, 0, k, LBM_NACC(a)), vR);
      if (NS > 2) acc_put<DET>(a.A_cur, LBM_OFF(a, kChkAcc, 0, a.acc_row + k, LBM_NACC(a)), vP);
    } else if (DET) {
      iR += acc_from(vR);
      if (NS > 2) iP += acc_from(vP);
    } else {
      fR = __fadd_rn(fR, vR);
      if (NS > 2) fP = __fadd_rn(fP, vP);
    }
  }
  if (!RS) {
    if (DET) {
      static_cast<acc_t *>(a.A_cur)[LBM_OFF(a, kChkAcc, 0, n, LBM_NACC(a))] = iR;
      if (NS > 2) static_cast<acc_t *>(a.A_cur)[LBM_OFF(a, kChkAcc, 0, a.acc_row + n, LBM_NACC(a))] = iP;
    } else {
      static_cast<float *>(a.A_cur)[LBM_OFF(a, kChkAcc, 0, n, LBM_NACC(a))] = fR;
      if (NS > 2) static_cast<float *>(a.A_cur)[LBM_OFF(a, kChkAcc, 0, a.acc_row + n, LBM_NACC(a))] = fP;
    }
  }
}

// Block-wide FP64 sum of K per-thread values, fixed order; result valid in
// thread 0. Must be called by every thread of the block.
template <int K>
__device__ __forceinline__ void block_sum_d(const float (&v)[K], double (&out)[K]) {
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

// Node block blk (nodes blk 256 .. blk 256 + 255) of a node kernel: the
// emission (banking the previous hits into the block's FP64 slot) or the
// hits. Every thread of the block must call it.
template <int ST, int LAYOUT, int NS, bool DET, bool RS, bool EMIT>
__device__ __forceinline__ void node_block(const StepArgs &a, int blk, int64_t t) {
  if ((int64_t)blk * kBlock >= a.n_nodes) return;  // (uniform over the block)
  const int64_t n = (int64_t)blk * kBlock + threadIdx.x;
  if (!EMIT) {
    if (n < a.n_nodes) node_hits<ST, LAYOUT, NS, DET, RS>(a, n, t);
    return;
  }
  float hv[2] = {0.f, 0.f};
  if (n < a.n_nodes) {
    node_emit<ST, LAYOUT, NS, DET, RS>(a, n, t, hv);
    if (n < a.bank_lo || n >= a.bank_hi) hv[0] = hv[1] = 0.f;  // (halo nodes are the neighbour's)
  }
  double hs[2];
  block_sum_d<2>(hv, hs);
  if (threadIdx.x == 0) {
    a.node_cum[2 * (int64_t)blk + 0] += hs[0];
    a.node_cum[2 * (int64_t)blk + 1] += hs[1];
  }
}

template <int ST, int LAYOUT, int NS, bool DET, bool RS, bool EMIT>
__global__ void __launch_bounds__(kBlock) node_kernel(const StepArgs a) {
  node_block<ST, LAYOUT, NS, DET, RS, EMIT>(a, (int)blockIdx.x, a.t);
}

// Fast kernel: one warp per listed lattice warp. These warps need no
// neighbour mask, no wall-hit accumulators and no face flows; even steps
// touch only the entries' own slots. Even steps take the whole fast list in
// one launch. Odd steps take it in two: the region warps at its head (UNI:
// cell = entry + the region's shift, a word of the small table after the
// lists, which stays in L1; no fcell, idx or nbm reads), then the rest.
template <int ST, int LAYOUT, int NS, int ODD, int PHYS, bool UNI = false>
__global__ void __launch_bounds__(kBlock, fast_min_blocks(ST, ODD)) fast_step_kernel(const StepArgs a) {
  const int w = (ODD && !UNI ? a.n_uni : 0) + (int)blockIdx.x * kWarpsPerBlock + (int)(threadIdx.x >> 5);
  if (w >= (UNI ? a.n_uni : a.n_fast + a.n_wall)) return;
  const uint32_t v = (uint32_t)__ldg(a.fast_list + w);
  const int32_t L = (int32_t)(v & kWarpIdMask) * 32 + (threadIdx.x & 31);
  if (L >= a.n_lat) return;
  int32_t cell = L;
  if (LAYOUT == LBM_LAYOUT_DENSE) {
    if (__ldg(a.mask + L)) return;
  } else if (UNI) {
    cell = L + __ldg(a.fast_list + a.n_lat_warps + ((v >> kUniShift) & (uint32_t)kUniRegions));
  } else if (ODD) {
    cell = __ldg(a.fcell + L);
  }
  float flux[6];
  // odd steps: one code path for plain and wall warps, the solid-neighbour
  // mask being zero for a plain warp (two paths in one kernel spill more)
  const uint32_t nbm = (ODD && !UNI && (v & kWallWarp)) ? __ldg(a.nbm + L) : 0u;
  cell_update<ST, LAYOUT, NS, ODD, false, true, false, PHYS, ODD != 0 && !UNI, true, UNI>(a, L, cell, nbm, a.t,
                                                                                        flux);
}

// General kernel: one warp per listed lattice warp (solid neighbours,
// inlet/outlet planes, halo planes).
template <int ST, int LAYOUT, int NS, int ODD, bool DET, bool RS, int PHYS>
__global__ void __launch_bounds__(kBlock, kGenMinBlocks) gen_step_kernel(const StepArgs a) {
  const int w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (w < a.n_gen) {
    const int32_t W = __ldg(a.gen_list + w);
    const int32_t L = W * 32 + (threadIdx.x & 31);
    float flux[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // in C,R,P ; out C,R,P
    if (L < a.n_lat) {
      const int32_t cell = (LAYOUT == LBM_LAYOUT_DENSE) ? L : __ldg(a.fcell + L);
      if ((LAYOUT != LBM_LAYOUT_DENSE || !__ldg(a.mask + cell)) && !halo_plane(a, cell / (a.nx * a.ny)))
        cell_update<ST, LAYOUT, NS, ODD, DET, false, RS, PHYS>(a, L, cell, __ldg(a.nbm + L), a.t, flux);
    }
    bank_flux(a, W, flux);
  }
}

// One step of the cells of one 256-entry block of lattice entries
// (single-launch batches): each warp takes the fast path when all its live
// entries can. Same arithmetic and face-flow slots as the fast and general
// kernels.
template <int ST, int LAYOUT, int NS, int ODD, bool DET, bool RS, int PHYS>
__device__ __forceinline__ void step_block(const StepArgs &a, const int blk, const int64_t t) {
  const int32_t L = (int32_t)(blk * kBlock + threadIdx.x);
  float flux[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // in C,R,P ; out C,R,P
  bool live = L < a.n_lat;
  int32_t cell = 0;
  uint32_t nbm = 0;
  if (live) {
    cell = (LAYOUT == LBM_LAYOUT_DENSE) ? L : __ldg(a.fcell + L);
    if (LAYOUT == LBM_LAYOUT_DENSE && __ldg(a.mask + cell)) live = false;
    nbm = __ldg(a.nbm + L);
  }
  // (halo cells are not stepped, and a warp holding one takes the general
  // path, as the warp lists have it)
  const bool halo = live && halo_plane(a, cell / (a.nx * a.ny));
  const bool plain = !live || (!halo && fast_entry(a, cell, nbm));
  const bool onplane = !live || (!halo && fast_plane(a, cell));
  live = live && !halo;
  if (__all_sync(0xffffffffu, plain) || (!ODD && __all_sync(0xffffffffu, onplane))) {
    if (live) cell_update<ST, LAYOUT, NS, ODD, DET, true, RS, PHYS>(a, L, cell, 0u, t, flux);
  } else if (__all_sync(0xffffffffu, onplane)) {  // a wall warp, odd step
    if (live) cell_update<ST, LAYOUT, NS, ODD, DET, true, RS, PHYS, true>(a, L, cell, nbm, t, flux);
  } else if (live) {
    cell_update<ST, LAYOUT, NS, ODD, DET, false, RS, PHYS>(a, L, cell, nbm, t, flux);
  }
  bank_flux(a, (int32_t)(L >> 5), flux);
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

// One launch covers p.n_steps steps in 3 n_steps phases of total_blocks
// CTAs, one work block each: for each step the node emission, the cell
// updates and the node hits (a simulation's n_blocks cover both its lattice
// blocks and its node blocks). A CTA takes the next ticket when it starts
// (ticket = phase x total_blocks + work block), and a CTA of phase k > 0
// first waits until every work block of phase k - 1 has finished: each
// phase reads what the previous one wrote. Tickets follow the order in
// which CTAs actually start, so every CTA a waiter depends on is already
// running or done, and the lowest unfinished phase never waits: the launch
// needs no co-residency guarantee. Each CTA runs exactly one work block,
// with no loop around the step (a loop of steps inside one CTA made the
// compiler spill about 1 KB per thread).
template <int ST, int LAYOUT, int NS, bool DET, bool RS, int PHYS>
__global__ void __launch_bounds__(kBlock, kGenMinBlocks) batch_step_kernel(const __grid_constant__ BatchLaunch p) {
  __shared__ int s_ticket;
  if (threadIdx.x == 0) {
    int tk = (int)atomicAdd(&p.sync->ticket, 1u);
    const int k = tk / p.total_blocks;
    if (*(volatile int *)&p.sync->timed_out ||
        (k > 0 &&
         !wait_counter(&p.sync->done[k - 1], (unsigned)p.total_blocks, &p.sync->timed_out, kWaitTimeoutNs)))
      tk = -1;
    s_ticket = tk;
  }
  __syncthreads();
  const int t = s_ticket;
  if (t < 0) return;  // a wait gave up: the host reports it
  const int ph = t / p.total_blocks;
  const int w = t - ph * p.total_blocks;
  const int ks = p.k0 + ph / 3;
  const int q = batch_sim_of(p, w);
  const StepArgs &a = p.v[q][ks % 6];
  const int64_t step = p.t0[q] + ks;
  const int blk = w - p.block_start[q];
  if (ph % 3 == 1) {
    if (a.parity)
      step_block<ST, LAYOUT, NS, 1, DET, RS, PHYS>(a, blk, step);
    else
      step_block<ST, LAYOUT, NS, 0, DET, RS, PHYS>(a, blk, step);
  } else if (!a.sp_bb) {
    if (ph % 3 == 0)
      node_block<ST, LAYOUT, NS, DET, RS, true>(a, blk, step);
    else
      node_block<ST, LAYOUT, NS, DET, RS, false>(a, blk, step);
  }
  __syncthreads();  // every thread's writes of this block precede the release
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&p.sync->done[ph], 1u);
  }
}

// Simulation whose blocks [start[k], start[k + 1]) hold block w.
__device__ __forceinline__ int batch_owner(const int32_t *start, int n, int w) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Per-step batched node kernels: node block w - node_start[q] of simulation
// q, each at its own step.
template <int ST, int LAYOUT, int NS, bool DET, bool RS, bool EMIT>
__global__ void __launch_bounds__(kBlock) batch_node_kernel(const __grid_constant__ BatchLaunch p) {
  const int w = (int)blockIdx.x;
  const int q = batch_owner(p.node_start, p.n_sims, w);
  const StepArgs &a = p.v[q][p.k0 % 6];
  if (a.sp_bb) return;
  node_block<ST, LAYOUT, NS, DET, RS, EMIT>(a, w - p.node_start[q], p.t0[q] + p.k0);
}

// Per-step batched launches, split as for a single simulation: the fast
// warps of every simulation in p, in two launches (the simulations at an
// even step, then those at an odd one: each launch has its parity's register
// budget), then the general warps. Same arithmetic and face-flow slots as
// the single-simulation kernels, so a simulation evolves identically alone
// or batched.
template <int ST, int LAYOUT, int NS, int PHYS, int ODD>
__global__ void __launch_bounds__(kBlock, fast_min_blocks(ST, ODD)) batch_fast_kernel(const __grid_constant__ BatchLaunch p) {
  const int w = (int)blockIdx.x;
  const int q = batch_owner(p.fast_start, p.n_sims, w);
  const StepArgs &a = p.v[q][p.k0 % 6];
  if (a.parity != ODD) return;  // (the other launch takes this simulation)
  const int64_t step = p.t0[q] + p.k0;
  const int lw = (w - p.fast_start[q]) * kWarpsPerBlock + (int)(threadIdx.x >> 5);
  if (lw >= a.n_fast + a.n_wall) return;
  // (region warps take the indexed addressing here, as the other warps do)
  const uint32_t v = (uint32_t)__ldg(a.fast_list + lw);
  const int32_t L = (int32_t)(v & kWarpIdMask) * 32 + (int32_t)(threadIdx.x & 31);
  if (L >= a.n_lat) return;
  int32_t cell = L;
  if (LAYOUT == LBM_LAYOUT_DENSE) {
    if (__ldg(a.mask + L)) return;
  } else if (ODD) {
    cell = __ldg(a.fcell + L);
  }
  float flux[6];
  const uint32_t nbm = (ODD && (v & kWallWarp)) ? __ldg(a.nbm + L) : 0u;
  cell_update<ST, LAYOUT, NS, ODD, false, true, false, PHYS, ODD != 0, true>(a, L, cell, nbm, step, flux);
}

template <int ST, int LAYOUT, int NS, bool DET, bool RS, int PHYS>
__global__ void __launch_bounds__(kBlock, kGenMinBlocks) batch_gen_kernel(const __grid_constant__ BatchLaunch p) {
  const int w = (int)blockIdx.x;
  const int q = batch_owner(p.gen_start, p.n_sims, w);
  const StepArgs &a = p.v[q][p.k0 % 6];
  const int64_t step = p.t0[q] + p.k0;
  const int blk = w - p.gen_start[q];
  const int lw = blk * kWarpsPerBlock + (int)(threadIdx.x >> 5);
  if (lw < a.n_gen) {
    const int32_t W = __ldg(a.gen_list + lw);
    const int32_t L = W * 32 + (int32_t)(threadIdx.x & 31);
    float flux[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (L < a.n_lat) {
      const int32_t cell = (LAYOUT == LBM_LAYOUT_DENSE) ? L : __ldg(a.fcell + L);
      if ((LAYOUT != LBM_LAYOUT_DENSE || !__ldg(a.mask + cell)) && !halo_plane(a, cell / (a.nx * a.ny))) {
        if (a.parity)
          cell_update<ST, LAYOUT, NS, 1, DET, false, RS, PHYS>(a, L, cell, __ldg(a.nbm + L), step, flux);
        else
          cell_update<ST, LAYOUT, NS, 0, DET, false, RS, PHYS>(a, L, cell, __ldg(a.nbm + L), step, flux);
      }
    }
    bank_flux(a, W, flux);
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
  const bool bc = (!a.periodic_z && (z == 0 || z == a.nz - 1)) || halo_plane(a, z);
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
  if ((!a.periodic_z && (z == 0 || z == a.nz - 1)) || halo_plane(a, z)) return;
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
// layout and species count only (LY, NSC)
#define LBM_DISPATCH_LN(LAYOUT_, NS_, ...)                                      \
  do {                                                                          \
    if ((LAYOUT_) == LBM_LAYOUT_DENSE) {                                        \
      constexpr int LY = LBM_LAYOUT_DENSE;                                      \
      if ((NS_) == 2) { constexpr int NSC = 2; __VA_ARGS__; }                   \
      else { constexpr int NSC = 3; __VA_ARGS__; }                              \
    } else {                                                                    \
      constexpr int LY = LBM_LAYOUT_FLUID;                                      \
      if ((NS_) == 2) { constexpr int NSC = 2; __VA_ARGS__; }                   \
      else { constexpr int NSC = 3; __VA_ARGS__; }                              \
    }                                                                           \
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
cudaError_t launch_step_st(const StepArgs &a, int layout, int ns, int parity, cudaStream_t st, const cudaEvent_t *ev) {
  if (ev) cudaEventRecord(ev[0], st);
  const unsigned ggrid = (unsigned)((a.n_gen + kWarpsPerBlock - 1) / kWarpsPerBlock);
  const unsigned ngrid = a.sp_bb ? 0u : (unsigned)((a.n_nodes + kBlock - 1) / kBlock);
  if (ngrid > 0) {
    LBM_DISPATCH_LNS(layout, ns, 0, a.det, node_kernel<ST, LY, NSC, DT, RS, true><<<ngrid, kBlock, 0, st>>>(a));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[1], st);
  // even steps: the whole fast list in one launch; odd steps: the region
  // warps (fluid-only addressing), then the plain and wall warps in
  // increasing order
  const int32_t n_uni = (parity && layout == LBM_LAYOUT_FLUID) ? a.n_uni : 0;
  if (n_uni > 0) {
    const unsigned ugrid = (unsigned)((n_uni + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (ns == 2)
      fast_step_kernel<ST, LBM_LAYOUT_FLUID, 2, 1, PHYS, true><<<ugrid, kBlock, 0, st>>>(a);
    else
      fast_step_kernel<ST, LBM_LAYOUT_FLUID, 3, 1, PHYS, true><<<ugrid, kBlock, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const unsigned fgrid =
      (unsigned)(((int64_t)a.n_fast + a.n_wall - n_uni + kWarpsPerBlock - 1) / kWarpsPerBlock);
  if (fgrid > 0) {
    if (parity)
      LBM_DISPATCH_LN(layout, ns, fast_step_kernel<ST, LY, NSC, 1, PHYS><<<fgrid, kBlock, 0, st>>>(a));
    else
      LBM_DISPATCH_LN(layout, ns, fast_step_kernel<ST, LY, NSC, 0, PHYS><<<fgrid, kBlock, 0, st>>>(a));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[2], st);
  if (ggrid > 0) {
    LBM_DISPATCH_LNS(layout, ns, parity, a.det, gen_step_kernel<ST, LY, NSC, OD, DT, RS, PHYS><<<ggrid, kBlock, 0, st>>>(a));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[3], st);
  if (ngrid > 0)
    LBM_DISPATCH_LNS(layout, ns, 0, a.det, node_kernel<ST, LY, NSC, DT, RS, false><<<ngrid, kBlock, 0, st>>>(a));
  if (ev) cudaEventRecord(ev[4], st);
  return cudaGetLastError();
}

template <int ST, bool RS, int PHYS>
cudaError_t launch_batch_st(const BatchLaunch &p, int layout, int ns, int det, cudaStream_t st) {
  if (p.total_blocks <= 0 || p.n_sims <= 0 || p.n_steps <= 0) return cudaSuccess;
  if (!p.sync || p.n_steps > kStepsPerLaunch) return cudaErrorInvalidValue;
  if (3 * (int64_t)p.n_steps * p.total_blocks >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)(3 * p.n_steps * p.total_blocks);
  LBM_DISPATCH_LNS(layout, ns, 0, det, batch_step_kernel<ST, LY, NSC, DT, RS, PHYS><<<grid, kBlock, 0, st>>>(p));
  return cudaGetLastError();
}

template <int ST, bool RS, int PHYS>
cudaError_t launch_batch_split_st(const BatchLaunch &p, int layout, int ns, int det, cudaStream_t st) {
  if (p.n_sims <= 0 || p.n_steps != 1) return cudaErrorInvalidValue;
  if (p.total_node > 0) {
    LBM_DISPATCH_LNS(layout, ns, 0, det,
                     batch_node_kernel<ST, LY, NSC, DT, RS, true><<<(unsigned)p.total_node, kBlock, 0, st>>>(p));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (p.total_fast > 0) {  // one launch per parity, each skipping the other parity's simulations
    LBM_DISPATCH_LN(layout, ns, batch_fast_kernel<ST, LY, NSC, PHYS, 0><<<(unsigned)p.total_fast, kBlock, 0, st>>>(p));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    LBM_DISPATCH_LN(layout, ns, batch_fast_kernel<ST, LY, NSC, PHYS, 1><<<(unsigned)p.total_fast, kBlock, 0, st>>>(p));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (p.total_gen > 0) {
    LBM_DISPATCH_LNS(layout, ns, 0, det,
                     batch_gen_kernel<ST, LY, NSC, DT, RS, PHYS><<<(unsigned)p.total_gen, kBlock, 0, st>>>(p));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (p.total_node > 0)
    LBM_DISPATCH_LNS(layout, ns, 0, det,
                     batch_node_kernel<ST, LY, NSC, DT, RS, false><<<(unsigned)p.total_node, kBlock, 0, st>>>(p));
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
  template cudaError_t launch_step_st<ST, RS, PHYS>(const StepArgs &, int, int, int, cudaStream_t, const cudaEvent_t *); \
  template cudaError_t launch_batch_st<ST, RS, PHYS>(const BatchLaunch &, int, int, int, cudaStream_t);   \
  template cudaError_t launch_batch_split_st<ST, RS, PHYS>(const BatchLaunch &, int, int, int, cudaStream_t);
#define LBM_INSTANTIATE_STORAGE(ST)                                                                    \
  LBM_INSTANTIATE_STEP(ST, false, kPhysCarrier)                                                               \
  template cudaError_t launch_plane_sums_st<ST>(const ObsArgs &, int, int, cudaStream_t);             \
  template cudaError_t launch_export_st<ST>(const StepArgs &, int, int, int, int, float *, cudaStream_t);

}  // namespace lbm
