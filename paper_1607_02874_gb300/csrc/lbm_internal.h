// Internal declarations shared by the liblbm translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>

#include "../../include/lbm.h"

namespace lbm {

constexpr int kQ = 19;
constexpr int kBlock = 256;
// Resident blocks per SM (256 threads each) that the register budgets of
// the step kernels aim at: the fast kernel (the warps away from the
// inlet/outlet and halo planes), per storage and parity, and the general
// kernel (every other warp) and the single-launch batched kernel.
// Measured on the 256x256x512 and 512x512x1024 C+R+P boxes: 16-bit even
// steps are 2% faster at 4 blocks (64 registers) than at 3. With the odd
// step's offsets in shared memory, 16-bit odd steps are 4% faster at 4
// blocks (64 registers, 16 bytes of spill) than at 3, and FP32 odd steps
// fastest at 3 (80 registers, no spill; 4 blocks spill 84 bytes and are 1%
// slower). The general kernel is slower at 3 than at 2 in both storages.
#ifndef LBM_FAST_EVEN_MINB
#define LBM_FAST_EVEN_MINB 4
#endif
#ifndef LBM_FAST_EVEN_MINB_F32
#define LBM_FAST_EVEN_MINB_F32 3
#endif
#ifndef LBM_FAST_ODD_MINB
#define LBM_FAST_ODD_MINB 4
#endif
#ifndef LBM_FAST_ODD_MINB_F32
#define LBM_FAST_ODD_MINB_F32 3
#endif
#ifndef LBM_GEN_MINB
#define LBM_GEN_MINB 2
#endif
constexpr int kGenMinBlocks = LBM_GEN_MINB;

constexpr int fast_min_blocks(int st, int odd) {
  return odd ? (st == LBM_FP32 ? LBM_FAST_ODD_MINB_F32 : LBM_FAST_ODD_MINB)
             : (st == LBM_FP32 ? LBM_FAST_EVEN_MINB_F32 : LBM_FAST_EVEN_MINB);
}
constexpr int kWarpsPerBlock = kBlock / 32;
// Entries of the fast kernel's warp list: the lattice warp number in the low
// 26 bits (lattice entries are int32, so at most 2^26 warps), a region
// number in bits 26-30 and the wall mark in bit 31. Region r > 0 marks a
// plain warp whose 32 entries and all their 18 neighbours are numbered in
// cell order with one shift D_r = cell - entry (in practice the all-fluid
// planes away from the porous sample). The region warps head the list
// (n_uni of them), and their odd steps run in a launch of their own that
// forms cells and neighbour entries by arithmetic instead of reading fcell
// and idx. The table of the D_r follows the lists (kUniTable words from
// word n_lat_warps; word 0 unused).
constexpr uint32_t kWallWarp = 0x80000000u;  // wall warp
constexpr int kUniShift = 26;
constexpr uint32_t kWarpIdMask = (1u << kUniShift) - 1u;
constexpr int kUniRegions = 31;
constexpr int kUniTable = kUniRegions + 1;

// D3Q19 speeds in the order documented in lbm.h. Written as constexpr
// functions so that fully unrolled loops fold them into immediates.
__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                : 0;
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1
                                                               : 0;
}
__host__ __device__ constexpr int cz(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// weights 1/3, 1/18, 1/36 and their exact reciprocals
__host__ __device__ constexpr float wq(int i) {
  return i == 0 ? (1.0f / 3.0f) : (i <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}
__host__ __device__ constexpr float inv_wq(int i) { return i == 0 ? 3.0f : (i <= 6 ? 18.0f : 36.0f); }

// Population storage. Every format holds the scaled deviation from the rest
// state, d_i = (f_i - w_i rho_ref) / w_i with rho_ref = 1 for the carrier and
// 0 for the species: O(1) numbers that keep the carrier density deviation
// (~1e-3) at full relative precision. (A reference density for the reactant
// would make the values near it small, but lose relative precision where
// the reactant is depleted, at the catalytic walls, whose hits make the
// product.) Collisions run in FP32.
//
// Two arrays: the carrier (one value per entry and slot) and the species
// (the reactant alone, or the reactant and product of one entry and slot as
// an adjacent pair, so that one 4-byte (16-bit formats) or 8-byte (FP32)
// access moves both). Pop<ST, NS> names the element types and the
// conversions between storage and FP32:
//   - FP32 stores d;
//   - FP16 stores the carrier rounded to nearest and the species, scaled by
//     the exact factor 2^14, rounded stochastically (concentrations down to
//     ~4e-9 stay in the normal range, values up to ~4 below the maximum);
//   - BF16 rounds every array stochastically.
// Stochastic rounding is unbiased where round-to-nearest is not: near
// equilibrium the populations of a region sit at nearly the same value and
// would round the same way every step, so a concentration field would
// freeze onto the format's grid and lose or gain mass coherently. It uses
// the conversion with explicit random bits (cvt.rs): for a pair, bits 0-12
// (binary16) or 0-15 (bfloat16) of the 32-bit word round the low element and
// bits 16-28 / 16-31 the high one; a lone value is converted as the low
// element. The words come from a counter-based hash of (entry, step) times a
// distinct odd constant per slot, so runs are reproducible.
// The species arithmetic runs in the stored (for FP16, 2^14-scaled) units:
// the species update is linear in the species values, so only the wall hits,
// the face flows, the plane cache and the observables convert.
template <int ST, int NS>
struct Pop;

template <int NS>
struct Pop<LBM_FP32, NS> {
  using C = float;
  using S = typename std::conditional<NS == 3, float2, float>::type;
  static constexpr float kSp = 1.0f, kSpInv = 1.0f;
  __device__ __forceinline__ static float c_val(C q) { return q; }
  __device__ __forceinline__ static float2 s_val(S q) {
    if constexpr (NS == 3) return q; else return make_float2(q, 0.0f);
  }
  __device__ __forceinline__ static C c_cv(float v, uint32_t) { return v; }
  __device__ __forceinline__ static S s_cv(float2 v, uint32_t) {
    if constexpr (NS == 3) return v; else return v.x;
  }
};

__device__ __forceinline__ uint32_t cvt_rs_f16x2(float hi, float lo, uint32_t r) {
  uint32_t d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
  return d;
}
__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float hi, float lo, uint32_t r) {
  uint32_t d;
  asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
  return d;
}

template <int NS>
struct Pop<LBM_FP16_DEV, NS> {
  using C = unsigned short;
  using S = typename std::conditional<NS == 3, unsigned, unsigned short>::type;
  static constexpr float kSp = 16384.0f, kSpInv = 1.0f / 16384.0f;  // 2^14, exact
  __device__ __forceinline__ static float c_val(C q) { return __half2float(__ushort_as_half(q)); }
  __device__ __forceinline__ static float2 s_val(S q) {
    if constexpr (NS == 3) {
      __half2 h;
      memcpy(&h, &q, 4);
      return __half22float2(h);
    } else {
      return make_float2(__half2float(__ushort_as_half(q)), 0.0f);
    }
  }
  __device__ __forceinline__ static C c_cv(float v, uint32_t) { return __half_as_ushort(__float2half_rn(v)); }
  __device__ __forceinline__ static S s_cv(float2 v, uint32_t r) {
    if constexpr (NS == 3) return cvt_rs_f16x2(v.y, v.x, r);
    else return (unsigned short)cvt_rs_f16x2(0.0f, v.x, r);
  }
};

template <int NS>
struct Pop<LBM_BF16_DEV, NS> {
  using C = unsigned short;
  using S = typename std::conditional<NS == 3, unsigned, unsigned short>::type;
  static constexpr float kSp = 1.0f, kSpInv = 1.0f;
  __device__ __forceinline__ static float c_val(C q) { return __uint_as_float((uint32_t)q << 16); }
  __device__ __forceinline__ static float2 s_val(S q) {
    if constexpr (NS == 3) return make_float2(__uint_as_float(q << 16), __uint_as_float(q & 0xffff0000u));
    else return make_float2(__uint_as_float((uint32_t)q << 16), 0.0f);
  }
  __device__ __forceinline__ static C c_cv(float v, uint32_t r) { return (unsigned short)cvt_rs_bf16x2(0.0f, v, r); }
  __device__ __forceinline__ static S s_cv(float2 v, uint32_t r) {
    if constexpr (NS == 3) return cvt_rs_bf16x2(v.y, v.x, r);
    else return (unsigned short)cvt_rs_bf16x2(0.0f, v.x, r);
  }
};

// Counter-based hashing for the stochastic rounding: the 32-bit finaliser of
// MurmurHash3 (Appleby) for the per-(entry, step) word, then one multiply by
// a distinct odd constant (golden-ratio Weyl sequence) per slot and array.
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__host__ __device__ constexpr uint32_t sr_mul(int array, int i) {
  return (0x9E3779B9u * (uint32_t)(2 * (array * 19 + i) + 1)) | 1u;
}

inline size_t storage_bytes(int st) { return st == LBM_FP32 ? 4 : 2; }
// Bytes of the carrier array (the species array follows it in the same
// allocation): 19 slots of n_pad entries.
inline size_t carrier_bytes(int64_t n_pad, int st) { return (size_t)kQ * n_pad * storage_bytes(st); }

// Round n up to a multiple of 64 entries (keeps every population row
// 128-byte aligned for 16-bit storage and 256-byte aligned for FP32).
inline int64_t pad64(int64_t n) { return (n + 63) / 64 * 64; }

struct DevAlloc {
  lbm_allocator a{};
  bool has = false;
  cudaStream_t stream = nullptr;
  void *alloc(size_t bytes);
  void free(void *p, size_t bytes);
};

// Wall hits accumulate as signed 64-bit fixed point with quantum 2^-58:
// integer addition is associative, so the sums (and every state downstream of
// them) do not depend on the order of the adds, and a simulation evolves
// bit-identically alone, inside a batched launch, or split into sub-domains
// whose cut nodes add the neighbour's share.
// Species populations are below 1 (concentrations <= c_in = 1), so the 18
// links of a node stay far inside the int64 range; values below 2^-58 are
// below any meaningful concentration.
// The conversions use only 32-bit float and integer operations (the 64-bit
// conversions and FP64 run on GB300's slow pipe): the high word is
// floor(v 2^26) and the low word the exact fractional remainder times 2^32,
// truncated. Only the observables widen to FP64.
using acc_t = unsigned long long;  // two's-complement bits of the int64 sum
__device__ __forceinline__ acc_t acc_from(float v) {
  const float x = v * 67108864.0f;                 // v 2^26, exact
  const float h = floorf(x);
  const int hi = __float2int_rz(h);                // exact: |h| < 2^31
  const unsigned lo = __float2uint_rz((x - h) * 4294967296.0f);  // remainder in [0, 1) times 2^32
  return ((acc_t)(unsigned)hi << 32) | (acc_t)lo;
}
__device__ __forceinline__ float acc_to_f(acc_t a) {
  const int hi = (int)(a >> 32);
  const unsigned lo = (unsigned)a;
  return fmaf(__uint2float_rn(lo), 3.4694469519536142e-18f /* 2^-58 */, __int2float_rn(hi) * 1.4901161193847656e-08f /* 2^-26 */);
}
__device__ __forceinline__ double acc_to_d(acc_t a) { return (double)(long long)a * 3.4694469519536142e-18; }

// Wall-hit accumulator of either kind: DET = fixed point (order-free),
// otherwise FP32 (summed by one thread per node in a fixed link order).
// k counts entries of the accumulator's own type.
template <bool DET>
__device__ __forceinline__ float acc_get(const void *A, int64_t k) {
  return DET ? acc_to_f(static_cast<const acc_t *>(A)[k]) : static_cast<const float *>(A)[k];
}
template <bool DET>
__device__ __forceinline__ double acc_get_d(const void *A, int64_t k) {
  return DET ? acc_to_d(static_cast<const acc_t *>(A)[k]) : (double)static_cast<const float *>(A)[k];
}
// Add v to slot k when one thread owns the slot (no atomics; the adds of
// that thread come in a fixed order).
template <bool DET>
__device__ __forceinline__ void acc_put(void *A, int64_t k, float v) {
  if (DET)
    static_cast<acc_t *>(A)[k] += acc_from(v);
  else
    static_cast<float *>(A)[k] = __fadd_rn(static_cast<float *>(A)[k], v);
}
template <bool DET>
__device__ __forceinline__ void acc_clear(void *A, int64_t k) {
  if (DET)
    static_cast<acc_t *>(A)[k] = 0ull;
  else
    static_cast<float *>(A)[k] = 0.0f;
}

// Unsigned division by an invariant divisor d (1 <= d < 2^31) as a
// multiply-high, a subtract, an add and two shifts (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994,
// Sec. 4): with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) for t = mulhi(m, n),
// exact for every 32-bit n.
struct FastDiv {
  uint32_t m;
  uint32_t s1, s2;
};
inline FastDiv fast_div_of(uint32_t d) {
  uint32_t l = 0;
  while (l < 32 && (1ull << l) < d) ++l;
  FastDiv f;
  f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1ull);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}
__device__ __forceinline__ uint32_t fast_div(uint32_t n, uint32_t m, uint32_t s1, uint32_t s2) {
  const uint32_t t = __umulhi(m, n);
  return (t + ((n - t) >> s1)) >> s2;
}

// Arguments of the fused step kernel and of the state readers (8-byte
// fields first, then 4-byte ones: 96 of these fill a batched launch's
// parameter space).
struct StepArgs {
  // --- pointers and 64-bit values ---
  void *f;               // carrier populations, warp-blocked [n_pad / 32][19][32] of Pop::C
  void *fs;              // species populations, warp-blocked [n_pad / 32][19][32] of Pop::S
  const uint8_t *mask;   // [n] 1 = solid
  const int32_t *idx;    // [n] lattice entry (fluid cells) / node number (catalytic solid) / -1
  const uint32_t *nbm;   // [n_lat] bit i: cell + c_i is a solid cell inside the box
  const int32_t *fcell;  // [n_lat] cell of each fluid entry (fluid-only layout)
  const float *inv_b;    // [n_nodes] 1 / b(node)
  const void *A_prev;    // [2][acc_row] species that reached the walls in the previous step (acc_t or float)
  void *A_cur;           // [2][acc_row] written by this step's node_hits_kernel
  void *A_next;          // [2][acc_row] the ring's third buffer (unused by the step)
  const float *ub_prev;  // [2 sides][5][plane] u and species rho of planes 1 / nz-2, previous step
  float *ub_cur;         // same, written this step
  double *node_cum;      // [node blocks][2] per-256-node-block cumulative sum of A_prev (R, P)
  double *flux_cum;      // [n_flux_slots][6] per-warp cumulative face flows (in C,R,P; out C,R,P)
  const int32_t *fast_list;  // [n_fast + n_wall] warps of the fast kernel (see kWallWarp), then the general
                             // list, then at word n_lat_warps the region shifts
  const int32_t *gen_list;   // [n_gen] every other warp with a live entry, increasing
  const int32_t *node_off;    // [n_nodes + 1] random matrix: first link slot of each node
  const uint32_t *cell_bits;  // [n] per solid cell: bit i set when cell + c_i is fluid
  const int32_t *node_cell;   // [n_nodes] the cell of each catalytic node
#ifdef LBM_CHECKED
  unsigned long long *check;  // first bounds violation (checked build only)
#endif
  int64_t n_pad;         // lattice entries rounded up to a multiple of 64
  int64_t n_lat;         // lattice entries (cells for dense, fluid cells for fluid-only)
  int64_t n_nodes;       // catalytic nodes
  int64_t t;             // the step this argument set advances (from t to t + 1)
  // wall-hit accumulators: species row stride of the ring buffers. Uniform
  // sputtering matrix: one value per node (the node count padded); random
  // matrix: one per active link of each node, the node's b links at
  // node_off[node] .. node_off[node + 1] - 1 in increasing direction
  // (the link count padded)
  int64_t acc_row;
  uint64_t rs_key;       // SplitMix64(seed) of the random matrix
  // --- 32-bit values ---
  int32_t nx, ny, nz;
  // division of a cell index by nx * ny and of the in-plane index by nx
  // through multiply-high (fast_div): multipliers and shifts (fast_div_of)
  uint32_t div_plane_m, div_nx_m, div_sh;
  int32_t periodic_z;
  int32_t n_lo_warps;    // lattice warps (32 entries) overlapping planes 0 and 1: flux slots 0..n_lo_warps-1
  int32_t hi_warp;       // first warp counted for the outlet side: max(first entry of plane nz-2 / 32, n_lo_warps)
  int32_t n_lat_warps;   // warps holding lattice entries
  int32_t n_fast, n_wall, n_gen;
  int32_t n_uni;         // region warps, at the head of fast_list and counted in n_fast
  float omega;           // relaxation rate of the carrier
  float c_in;
  float drho_in, drho_out;  // rho_in - 1, rho_out - 1 formed in double (full relative precision)
  float em_R;            // (1 - pS_R): reactant re-emission factor
  float em_PR;           // p pS_R: product from reactant
  float em_P;            // (1 - pS_P): product re-emission factor
  int32_t parity;        // t & 1 of the step this argument set advances (batched launches)
  int32_t det;           // wall hits in fixed point (1) or FP32 (0)
  uint32_t seed_mix;     // per-simulation part of the stochastic rounding's per-step seed
  int32_t rs;            // 1: random one-hot sputtering matrix
  int32_t bary;          // 1: every array relaxes towards the barycentric velocity
  int32_t vel_in;        // 1: the inlet plane takes the fixed velocity (0, 0, u_in)
  float u_in;
  float omega_s;         // relaxation rate of the reactant and product
  float g_z;             // body-force acceleration along z on the carrier (0: none)
  int32_t phys;          // kPhysCarrier, kPhysBary or kPhysChannel (the kernel variant)
  // z decomposition: planes 0, 1 (halo_lo) / nz-2, nz-1 (halo_hi) are a halo
  // copied from the neighbouring sub-domain (not stepped; no inlet/outlet
  // there); catalytic nodes [bank_lo, bank_hi) are this sub-domain's own
  // (the others, in halo planes, are not banked into the cumulative hits);
  // hash_base: added to the entry number in the stochastic-rounding hash
  int32_t halo_lo, halo_hi;
  uint32_t hash_base;
  int32_t bank_lo, bank_hi;
  int32_t sp_bb;         // 1: species bounce back at every solid (channel variant only)
};

// Neighbour cells of one cell (32-bit: boxes hold fewer than 2^31 cells).
struct Nbr {
  int32_t cell = 0, oxm = 0, oxp = 0, oym = 0, oyp = 0, ozm = 0, ozp = 0;
  Nbr() = default;
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

// Whether plane z is a halo plane of a sub-domain (never stepped).
__host__ __device__ __forceinline__ bool halo_plane(const StepArgs &a, int z) {
  return (a.halo_lo && z < 2) || (a.halo_hi && z >= a.nz - 2);
}
// Whether the cell lies away from the planes z = 0, 1, nz-2, nz-1, which take
// part in the inlet/outlet conditions or are halo planes (periodic z: the
// wrapping planes 0 and nz-1 are left to the general path, so that
// fast-kernel neighbours lie within two planes).
__device__ __forceinline__ bool fast_plane(const StepArgs &a, int32_t cell) {
  const int z = cell / (a.nx * a.ny);
  return a.periodic_z ? (z > 0 && z < a.nz - 1) : (z > 1 && z < a.nz - 2);
}
// Whether a fluid entry in cell `cell` with neighbour mask nbm is plain: no
// solid neighbour, on a fast plane. A warp whose live entries are all plain
// is a plain warp; one whose live entries are all on fast planes, some with
// a solid neighbour, is a wall warp. Both go to the fast kernel (wall warps
// with the halfway bounce-back's redirection on odd steps); every other warp
// to the general kernel.
__device__ __forceinline__ bool fast_entry(const StepArgs &a, int32_t cell, uint32_t nbm) {
  return nbm == 0 && fast_plane(a, cell);
}

// Checked build (-DLBM_CHECKED, a debugging aid where compute-sanitizer is
// not available): the population, accumulator, geometry-index and
// plane-cache accesses of the step and state-reading kernels are tested
// against their buffers' extents. The first violation is recorded in the
// device word a.check (kind in the top 8 bits, the element index below) and
// the access goes to element 0 of the same buffer instead, so nothing outside
// a buffer is touched. LBM_OFF(a, kind, base, off, limit) returns the offset
// off to add to a pointer at element base of a buffer of limit elements; the
// default build compiles it to off.
enum CheckKind { kChkPop = 1, kChkAcc = 2, kChkIdx = 3, kChkUb = 4, kChkNode = 5 };
#ifdef LBM_CHECKED
__device__ __forceinline__ int64_t lbm_chk(unsigned long long *word, int kind, int64_t base, int64_t off,
                                           int64_t limit) {
  const int64_t i = base + off;
  if (i >= 0 && i < limit) return off;
  atomicCAS(word, 0ull, ((unsigned long long)kind << 56) | ((unsigned long long)i & ((1ull << 56) - 1ull)));
  return -base;
}
#define LBM_OFF(a, kind, base, off, limit) \
  lbm_chk((a).check, (kind), (int64_t)(base), (int64_t)(off), (int64_t)(limit))
#else
#define LBM_OFF(a, kind, base, off, limit) (off)
#endif
// extents for the checks
#define LBM_NCELLS(a) ((int64_t)(a).nx * (a).ny * (a).nz)
#define LBM_NPOP(a) ((int64_t)kQ * (a).n_pad)
#define LBM_NACC(a) (2 * (a).acc_row)
#define LBM_NUB(a) ((int64_t)10 * (a).nx * (a).ny)

// Physics variants of the step kernels (a compile-time parameter):
//   kPhysCarrier  species follow the carrier velocity (default);
//   kPhysBary     every array relaxes towards the barycentric velocity;
//   kPhysChannel  carrier velocity plus the validation-channel ingredients:
//                 inert solid, body force, species relaxation time, and the
//                 species bounce-back mode.
constexpr int kPhysCarrier = 0, kPhysBary = 1, kPhysChannel = 2;

// SplitMix64 (Steele, Lea and Flood 2014): the first output for state x.
__host__ __device__ __forceinline__ uint64_t splitmix64_next(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Random sputtering matrix, one-hot columns: the outgoing link drawn for the
// population that reaches the catalytic node in cell `cell` along c_j at step
// t, as its rank r among the node's b active links (increasing direction).
// With h the high 32 bits of SplitMix64(key ^ (t 2^40 + cell 2^5 + j)),
// key = SplitMix64(seed), r = floor(h b / 2^32): uniform over the active
// links, so the mean matrix is S_ij = 1/b.
__device__ __forceinline__ int rs_rank(uint64_t key, int32_t cell, int j, int64_t t, int b) {
  const uint64_t k = ((uint64_t)t << 40) + ((uint64_t)(uint32_t)cell << 5) + (uint64_t)j;
  const uint64_t h = splitmix64_next(key ^ k) >> 32;
  return (int)((h * (uint64_t)b) >> 32);
}

// Seed of the stochastic rounding for the step that advances a simulation
// from time t: the high word of a Weyl step (golden-ratio increment) xor a
// per-simulation word. The host (single launches) and the batched kernel
// (which derives it per step) use this one definition.
__host__ __device__ __forceinline__ uint32_t step_seed_of(int64_t t, uint32_t seed_mix) {
  return (uint32_t)(((uint64_t)t * 0x9E3779B97F4A7C15ull) >> 32) ^ seed_mix;
}
__host__ __device__ __forceinline__ uint32_t seed_mix_of(uint64_t geometry_seed) {
  return (uint32_t)(geometry_seed * 0x85EBCA77u);
}

// Arguments of one batched launch, passed whole as a __grid_constant__
// kernel parameter so that every field is read from the constant bank (a
// copy in shared memory made the compiler hold the fields in registers and
// spill). Per simulation k: its arguments for the six steps t0_k .. t0_k + 5
// (the accumulator ring has period 3, the plane cache period 2, so step
// t0_k + j uses variant j mod 6 with its own rounding seed), its first block
// and t0_k. The launch advances steps k0 .. k0 + n_steps - 1 of the batch.
#ifdef LBM_CHECKED
constexpr int kMaxBatch = 12;  // (the checked build's StepArgs carry one more pointer)
#else
constexpr int kMaxBatch = 14;
#endif
struct BatchLaunch {
  StepArgs v[kMaxBatch][6];
  int64_t t0[kMaxBatch];
  int32_t block_start[kMaxBatch + 1];
  int32_t n_sims;
  int32_t total_blocks;
  int32_t k0;
  int32_t n_steps;
  struct BatchSync *sync;
  // per-step launches: blocks of the fast kernel (the fast warps) and of the
  // general kernel (the general warps and the catalytic nodes) of each
  // simulation, [fast_start[k], fast_start[k + 1]) and likewise
  int32_t fast_start[kMaxBatch + 1];
  int32_t gen_start[kMaxBatch + 1];
  int32_t node_start[kMaxBatch + 1];  // blocks of the two catalytic-node kernels (256 nodes each)
  int32_t total_fast, total_gen, total_node;
};
// Kernel parameters may hold up to 32,764 bytes (CUDA 12.1 and later). Measured
// on GB300 (CUDA 13.0): with argument blocks of 32,696 bytes every
// simulation after the first came out different from its run alone; blocks
// of 31,928 bytes (an earlier layout) and smaller agree bit for bit. So the
// arguments keep a margin below the documented limit.
static_assert(sizeof(BatchLaunch) <= 30720, "batched launch arguments too close to the kernel parameter limit");

// Launch one step of parity (t & 1) for the given storage/layout/species:
// the catalytic nodes' emission (node_emit_kernel), the fast kernel over
// a.fast_list, the general kernel over a.gen_list, then the nodes' wall
// hits (node_hits_kernel).
// ev (optional, measurement): five events, recorded before the emission,
// the fast kernel, the general kernel and the hits, and after the hits.
cudaError_t launch_step(const StepArgs &a, int storage, int layout, int ns, int parity, cudaStream_t st,
                        const cudaEvent_t *ev = nullptr);
// Per lattice warp: 0 no live entry, 1 plain, 2 general, 3 wall.
cudaError_t launch_warp_class(const StepArgs &a, int layout, uint8_t *cls, int32_t *shift, cudaStream_t st);
// RS: the random sputtering matrix; PHYS: the physics variant (kPhys*). Both
// are compile-time parameters, so that the default kernels carry none of the
// other variants' code; each combination other than the default is compiled
// in a translation unit of its own (step_*_rs.cu, step_*_bary.cu,
// step_*_rs_bary.cu, step_*_chan.cu, step_*_rs_chan.cu).
template <int ST, bool RS, int PHYS>
cudaError_t launch_step_st(const StepArgs &a, int layout, int ns, int parity, cudaStream_t st, const cudaEvent_t *ev);
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait of one thread until *ctr >= target. Gives up after timeout_ns
// of the global timer, after 2^28 polls whatever the timer says, or when
// *flag is already set; on giving up it sets *flag. Returns true when the
// count was reached. The acquire load orders the caller's later reads after
// the writes that the counted arrivals released.
__device__ __forceinline__ bool wait_counter(const unsigned *ctr, unsigned target, int *flag,
                                             unsigned long long timeout_ns) {
  const unsigned long long t0 = global_ns();
  unsigned polls = 0;
  while (ld_acquire_gpu(ctr) < target) {
    if (*(volatile int *)flag) return false;
    if (++polls >= (1u << 28) || ((polls & 63u) == 0 && global_ns() - t0 > timeout_ns)) {
      atomicExch(flag, 1);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// Limit of one wait inside a batched launch.
constexpr unsigned long long kWaitTimeoutNs = 2000000000ULL;
// Steps per multi-step batched launch.
constexpr int kStepsPerLaunch = 1024;

// Step ordering of a multi-step batched launch (zeroed before the launch):
// every CTA takes the next ticket, ticket -> (step, work block); a CTA of
// step k > 0 waits until done[k - 1] counts every work block of step k - 1.
struct BatchSync {
  unsigned ticket;
  int timed_out;
  unsigned done[3 * kStepsPerLaunch];  // per phase: node emission, cells, node hits of each step
};

// Batched launch (same storage, layout, species and accumulation mode for
// every simulation in p) of 3 p.n_steps x p.total_blocks CTAs: per step the
// node emission, the cell updates and the node hits, each phase after the
// previous one. With p.n_steps > 1, p.sync must point to a zeroed BatchSync.
template <int ST, bool RS, int PHYS>
cudaError_t launch_batch_st(const BatchLaunch &p, int layout, int ns, int det, cudaStream_t st);
// One step of every simulation in p (p.n_steps = 1) as four launches: the
// emission of all catalytic nodes, the fast warps of all, the general warps
// of all, then the wall hits of all nodes.
template <int ST, bool RS, int PHYS>
cudaError_t launch_batch_split_st(const BatchLaunch &p, int layout, int ns, int det, cudaStream_t st);

// Observables: per-plane FP64 sums [nz][kPlaneCols] = rhoC, rhoR, rhoP,
// rhoP*uz, hits R, hits P (last step).
constexpr int kPlaneCols = 6;
struct ObsArgs {
  StepArgs s;
  int parity;
  const int64_t *lat_plane;   // [nz+1] first lattice entry of each plane (device)
  const int64_t *node_plane;  // [nz+1] first node of each plane (device)
  double *plane_sums;         // [nz][kPlaneCols]
};
cudaError_t launch_plane_sums(const ObsArgs &a, int storage, int layout, int ns, cudaStream_t st);
template <int ST>
cudaError_t launch_plane_sums_st(const ObsArgs &a, int layout, int ns, cudaStream_t st);
// sum the columns of a row-major [rows][cols] FP64 array into out[cols], fixed order
cudaError_t launch_sum_columns(const double *in, int64_t rows, int cols, double *out, cudaStream_t st);
// dense field / population export at the current state
// which = LBM_FIELD_* or -1 for all populations [ns][19][n]
cudaError_t launch_export(const StepArgs &a, int parity, int storage, int layout, int ns, int which, float *dst,
                          cudaStream_t st);
template <int ST>
cudaError_t launch_export_st(const StepArgs &a, int parity, int layout, int ns, int which, float *dst,
                             cudaStream_t st);
cudaError_t launch_site_map(const void *A_prev_R, int det, int64_t n_nodes, const int32_t *node_off, float coef,
                            float *dst, cudaStream_t st);

// Geometry helpers.
void grf_mask(int nx, int ny, int nz, int z0, int z1, double porosity, double corr_len, uint64_t seed,
              uint8_t *mask);
double chord_length(int nx, int ny, int nz, int z0, int z1, const uint8_t *mask);

void set_error(const std::string &msg);

}  // namespace lbm

struct lbm_sim;
namespace lbm {
// Kernel arguments for the simulation's current step (capi.cu).
StepArgs make_args(const lbm_sim *s);
}  // namespace lbm

struct lbm_geometry {
  int32_t nx = 0, ny = 0, nz = 0, z0 = 0, z1 = 0, bc = 0;
  int32_t halo_lo = 0, halo_hi = 0, z_base = 0;  // z decomposition (lbm_geometry_desc)
  int64_t fluid_base = 0;
  uint64_t seed = 0;
  uint64_t mask_hash = 0;  // FNV-1a 64 of the solid mask (checkpoint compatibility)
  int64_t n = 0, plane = 0;
  int64_t n_fluid = 0, n_nodes = 0, n_links = 0;
  int64_t n_inert = 0;  // inert solid cells (mask value 2)
  double delta = 0.0;
  int device = 0;
  lbm::DevAlloc mem;
  uint8_t *mask = nullptr;      // [n]
  int32_t *idx = nullptr;       // [n]
  int32_t *b = nullptr;         // [n]
  uint32_t *nbm_dense = nullptr;  // [n] fluid cells: solid targets c + c_i; solid cells: fluid ones
  uint32_t *nbm_fluid = nullptr;  // [n_fluid]
  int32_t *fcell = nullptr;     // [n_fluid]
  int32_t *node_cell = nullptr;  // [n_nodes]
  float *inv_b = nullptr;       // [n_nodes]
  int64_t *fl_plane_d = nullptr, *cell_plane_d = nullptr, *node_plane_d = nullptr;  // [nz+1]
  int64_t *fl_plane_h = nullptr, *node_plane_h = nullptr;                            // host copies
};

struct lbm_sim {
  const lbm_geometry *g = nullptr;
  lbm_params prm{};
  int ns = 2, storage = LBM_FP32, layout = LBM_LAYOUT_DENSE, det = 0;
  double p = 1.0;
  int64_t t = 0;
  lbm::DevAlloc mem;
  int64_t n_lat = 0, n_pad = 0, n_nodes_pad = 0;
  void *f = nullptr;
  void *A = nullptr;        // [3][2][acc_row] wall-hit ring (8-byte slots; FP32 mode uses half)
  int64_t acc_row = 0;      // n_nodes_pad, or the padded link count with the random sputtering matrix
  int32_t *node_off = nullptr;  // [n_nodes + 1] random matrix: first link slot of each node
  int rs = 0;               // random sputtering matrix
  int bary = 0;             // barycentric velocity
  int phys = 0;             // kernel physics variant (kPhys*)
  int vel_in = 0;           // velocity inlet
  int sp_bb = 0;            // species bounce back at every solid
  float *ub = nullptr;      // [2][2][5][plane]
  double *node_cum = nullptr;
  int64_t n_blocks = 0;
  double *flux_cum = nullptr;
  int64_t n_flux_slots = 0;
  int32_t n_lo_warps = 0, hi_warp = 0, n_lat_warps = 0;
  int32_t *wlist = nullptr;  // fast list (region warps, then plain and wall warps), general list, region shifts
  int32_t n_fast = 0, n_wall = 0, n_gen = 0;
  int32_t n_uni = 0;  // region warps (kUniShift), counted among n_fast
  uint8_t last_warp_cls = 0;  // class of the (possibly partial) last lattice warp: 1 plain, 2 general, 3 wall
  double *plane_sums = nullptr;  // [nz][kPlaneCols]
  double *red_out = nullptr;     // [8]
  double M0[3] = {0, 0, 0};
  size_t bytes = 0;
};
