// Halo exchange between the sub-domains of a decomposition along z.
//
// Neighbouring sub-domains share two planes at each cut: a sub-domain's
// first real plane is its lower neighbour's inner halo plane, and the
// neighbour's last real plane is its own inner halo. With in-place (AA)
// streaming only odd steps reach across a plane: a cell of the real plane
// reads and writes slot k of its neighbour x + c_k. So, around an odd step:
//   - before it, the inner halo receives the slots of the neighbour's real
//     plane that point across the cut (c_z towards this sub-domain), which
//     the neighbour's even step wrote;
//   - after it, those slots of the inner halo, which this sub-domain's cells
//     wrote, go back into the neighbour's real plane (except where the cell
//     behind them, on the neighbour's side, is solid: there the neighbour
//     wrote its own bounce-back into the slot).
// Catalytic nodes of the two shared planes collect wall hits on both sides;
// after every step each side adds the other's hits, so that both hold the
// totals that the sputtering law re-emits one step later (the outer halo
// plane supplies the links that set b(x) of the inner plane's nodes). Only
// the nodes of a sub-domain's own planes are banked into its cumulative
// hits.
#include <algorithm>

#include "lbm_internal.h"

namespace lbm {
namespace {

// the five slots with c_z = +1 (up) or c_z = -1, in increasing order
__device__ __forceinline__ int cross_slot(int j, bool up) {
  const int u[5] = {5, 11, 14, 15, 18}, d[5] = {6, 12, 13, 16, 17};
  return up ? u[j] : d[j];
}

__device__ __forceinline__ int64_t ent_off_h(int32_t e) { return (int64_t)(e >> 5) * (kQ * 32) + (e & 31); }

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) / 16 * 16; }

// One thread per (slot j, entry e0 + i): buf holds [5][n] carrier values,
// then (from a 16-byte boundary) [5][n] species values.
template <typename CT, typename STy>
__global__ void halo_pops_kernel(const StepArgs a, int dense, int64_t e0, int64_t n, int up, int unpack,
                                 int check_upwind, char *buf) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5 * n) return;
  const int j = (int)(t / n);
  const int32_t e = (int32_t)(e0 + t % n);
  const int k = cross_slot(j, up != 0);
  CT *C = static_cast<CT *>(a.f);
  STy *S = static_cast<STy *>(a.fs);
  const int64_t off = ent_off_h(e) + 32 * k;
  CT *bc = reinterpret_cast<CT *>(buf);
  STy *bs = reinterpret_cast<STy *>(buf + align16(5 * (size_t)n * sizeof(CT)));
  if (!unpack) {
    bc[t] = C[off];
    bs[t] = S[off];
    return;
  }
  if (check_upwind) {
    const int32_t cell = dense ? e : a.fcell[e];
    const int32_t plane = a.nx * a.ny;
    const int z = cell / plane;
    const int32_t xy = cell - z * plane;
    const int y = xy / a.nx, x = xy - y * a.nx;
    const int xu = (x - cx(k) + a.nx) % a.nx, yu = (y - cy(k) + a.ny) % a.ny, zu = z - cz(k);
    if (a.mask[((int64_t)zu * a.ny + yu) * a.nx + xu]) return;  // the bounce-back written here stays
  }
  C[off] = bc[t];
  S[off] = bs[t];
}

// One thread per (species row r, node k0 + i) of the two shared planes:
// pack this step's hits, or add the neighbour's.
template <bool DET>
__global__ void halo_hits_kernel(const StepArgs a, int64_t k0, int64_t m, int rows, int unpack, char *buf) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * m) return;
  const int r = (int)(t / m);
  const int64_t idx = r * a.acc_row + k0 + t % m;
  if (DET) {
    acc_t *A = static_cast<acc_t *>(const_cast<void *>(a.A_prev));
    acc_t *b = reinterpret_cast<acc_t *>(buf);
    if (unpack)
      A[idx] += b[t];  // two's-complement fixed point: exact and order-free
    else
      b[t] = A[idx];
  } else {
    float *A = static_cast<float *>(const_cast<void *>(a.A_prev));
    float *b = reinterpret_cast<float *>(buf);
    if (unpack)
      A[idx] += b[t];
    else
      b[t] = A[idx];
  }
}

template <typename CT, typename STy>
cudaError_t launch_pops(const StepArgs &a, int dense, int64_t e0, int64_t n, int up, int unpack, int check, char *buf,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((5 * n + 255) / 256);
  halo_pops_kernel<CT, STy><<<grid, 256, 0, st>>>(a, dense, e0, n, up, unpack, check, buf);
  return cudaGetLastError();
}

// bytes of one side's population buffer for plane z: [5][n] carrier, [5][n] species
size_t pop_buffer_bytes(const lbm_sim *s, int64_t n) {
  const size_t sc = storage_bytes(s->storage);
  const size_t ss = sc * (s->ns == 3 ? 2 : 1);
  return align16(5 * (size_t)n * sc) + 5 * (size_t)n * ss;
}

int64_t plane_entries(const lbm_sim *s, int z, int64_t *first) {
  const lbm_geometry *g = s->g;
  if (s->layout == LBM_LAYOUT_DENSE) {
    *first = (int64_t)z * g->plane;
    return g->plane;
  }
  *first = g->fl_plane_h[z];
  return g->fl_plane_h[z + 1] - g->fl_plane_h[z];
}

bool halo_side_ok(const lbm_sim *s, int side) {
  if (!s || s->rs) return false;
  if (side == LBM_HALO_LO) return s->g->halo_lo != 0;
  if (side == LBM_HALO_HI) return s->g->halo_hi != 0;
  return false;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_halo_bytes(const lbm_sim *s, int side, size_t *pop_bytes, size_t *hit_bytes) {
  if (!halo_side_ok(s, side)) {
    set_error("no halo at that side of this simulation (or the random sputtering matrix, which has none)");
    return LBM_ERR_ARG;
  }
  const int nz = s->g->nz;
  const int zr = side == LBM_HALO_LO ? 2 : nz - 3, zh = side == LBM_HALO_LO ? 1 : nz - 2;
  int64_t f;
  if (pop_bytes)
    *pop_bytes = std::max(pop_buffer_bytes(s, plane_entries(s, zr, &f)), pop_buffer_bytes(s, plane_entries(s, zh, &f)));
  if (hit_bytes) {
    const int zlo = std::min(zr, zh);
    const int64_t m = s->g->node_plane_h[zlo + 2] - s->g->node_plane_h[zlo];
    *hit_bytes = (size_t)(s->ns - 1) * (size_t)m * (s->det ? sizeof(acc_t) : sizeof(float));
  }
  return LBM_OK;
}

extern "C" int lbm_halo_pops(lbm_sim *s, int side, int phase, int dir, void *buf) {
  if (!halo_side_ok(s, side) || !buf || (phase != LBM_HALO_PRE && phase != LBM_HALO_POST) ||
      (dir != LBM_HALO_PACK && dir != LBM_HALO_UNPACK)) {
    set_error("lbm_halo_pops: bad side, phase, direction or buffer");
    return LBM_ERR_ARG;
  }
  const int nz = s->g->nz;
  const bool lo = side == LBM_HALO_LO;
  const int zr = lo ? 2 : nz - 3, zh = lo ? 1 : nz - 2;
  // PRE: pack the real plane, unpack into the halo; POST: the reverse
  const bool real = (phase == LBM_HALO_PRE) == (dir == LBM_HALO_PACK);
  const int z = real ? zr : zh;
  // slots across the cut: the real plane's are those the neighbour's cells
  // reach (c_z from the neighbour into this sub-domain: up at the lower
  // cut), the halo's those this sub-domain's cells reach (down there)
  const int up = (real == lo) ? 1 : 0;
  const int check = phase == LBM_HALO_POST && dir == LBM_HALO_UNPACK;
  int64_t e0 = 0;
  const int64_t n = plane_entries(s, z, &e0);
  const StepArgs a = make_args(s);
  const int dense = s->layout == LBM_LAYOUT_DENSE;
  const int unpack = dir == LBM_HALO_UNPACK;
  char *b = static_cast<char *>(buf);
  cudaStream_t st = s->mem.stream;
  cudaError_t e;
  if (s->storage == LBM_FP32)
    e = s->ns == 3 ? launch_pops<float, float2>(a, dense, e0, n, up, unpack, check, b, st)
                   : launch_pops<float, float>(a, dense, e0, n, up, unpack, check, b, st);
  else
    e = s->ns == 3 ? launch_pops<unsigned short, unsigned>(a, dense, e0, n, up, unpack, check, b, st)
                   : launch_pops<unsigned short, unsigned short>(a, dense, e0, n, up, unpack, check, b, st);
  if (e != cudaSuccess) {
    set_error(std::string("halo populations: ") + cudaGetErrorString(e));
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}

extern "C" int lbm_halo_hits(lbm_sim *s, int side, int dir, void *buf) {
  if (!halo_side_ok(s, side) || !buf || (dir != LBM_HALO_PACK && dir != LBM_HALO_UNPACK)) {
    set_error("lbm_halo_hits: bad side, direction or buffer");
    return LBM_ERR_ARG;
  }
  const int nz = s->g->nz;
  const int zlo = side == LBM_HALO_LO ? 1 : nz - 3;  // the two shared planes
  const int64_t k0 = s->g->node_plane_h[zlo], m = s->g->node_plane_h[zlo + 2] - k0;
  if (m <= 0 || s->ns < 2) return LBM_OK;
  const StepArgs a = make_args(s);  // A_prev: the hits of the step just taken
  const int rows = s->ns - 1;
  const unsigned grid = (unsigned)((rows * m + 255) / 256);
  char *b = static_cast<char *>(buf);
  const int unpack = dir == LBM_HALO_UNPACK;
  if (s->det)
    halo_hits_kernel<true><<<grid, 256, 0, s->mem.stream>>>(a, k0, m, rows, unpack, b);
  else
    halo_hits_kernel<false><<<grid, 256, 0, s->mem.stream>>>(a, k0, m, rows, unpack, b);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("halo hits: ") + cudaGetErrorString(e));
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}
