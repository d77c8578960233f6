// C-ABI entry points of liblbm (declared in include/lbm.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm_internal.h"

namespace {
// An NVTX range around each public call (named after it), so that profilers
// attribute kernels to lbm_step, lbm_observables and so on; without a tool
// attached a range costs a predicted branch.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

namespace lbm {

cudaError_t build_structures(lbm_geometry *g, cudaStream_t st);

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

void *DevAlloc::alloc(size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (has) return a.alloc(a.ctx, bytes, (void *)stream);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void DevAlloc::free(void *p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 256;
  if (has)
    a.free(a.ctx, p, bytes, (void *)stream);
  else
    cudaFreeAsync(p, stream);
}

static int cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return LBM_ERR_CUDA;
}

static int arg_fail(const std::string &what) {
  set_error(what);
  return LBM_ERR_ARG;
}

#define LBM_CUDA_TRY(expr, what)              \
  do {                                        \
    cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// random sputtering matrix x physics variant, one storage type
template <int ST, bool RS>
static cudaError_t launch_step_phys(const StepArgs &a, int layout, int ns, int parity, cudaStream_t st,
                                   const cudaEvent_t *ev) {
  switch (a.phys) {
    case kPhysBary: return launch_step_st<ST, RS, kPhysBary>(a, layout, ns, parity, st, ev);
    case kPhysChannel: return launch_step_st<ST, RS, kPhysChannel>(a, layout, ns, parity, st, ev);
    default: return launch_step_st<ST, RS, kPhysCarrier>(a, layout, ns, parity, st, ev);
  }
}

template <int ST>
static cudaError_t launch_step_modes(const StepArgs &a, int layout, int ns, int parity, cudaStream_t st,
                                     const cudaEvent_t *ev) {
  return a.rs ? launch_step_phys<ST, true>(a, layout, ns, parity, st, ev)
              : launch_step_phys<ST, false>(a, layout, ns, parity, st, ev);
}

cudaError_t launch_step(const StepArgs &a, int storage, int layout, int ns, int parity, cudaStream_t st,
                        const cudaEvent_t *ev) {
  switch (storage) {
    case LBM_FP32: return launch_step_modes<LBM_FP32>(a, layout, ns, parity, st, ev);
    case LBM_FP16_DEV: return launch_step_modes<LBM_FP16_DEV>(a, layout, ns, parity, st, ev);
    default: return launch_step_modes<LBM_BF16_DEV>(a, layout, ns, parity, st, ev);
  }
}

template <int ST, bool RS>
static cudaError_t launch_batch_phys(const BatchLaunch &p, int layout, int ns, int det, cudaStream_t st) {
  switch (p.v[0][0].phys) {  // every simulation of a launch group has the same modes
    case kPhysBary: return launch_batch_st<ST, RS, kPhysBary>(p, layout, ns, det, st);
    case kPhysChannel: return launch_batch_st<ST, RS, kPhysChannel>(p, layout, ns, det, st);
    default: return launch_batch_st<ST, RS, kPhysCarrier>(p, layout, ns, det, st);
  }
}

template <int ST>
static cudaError_t launch_batch_modes(const BatchLaunch &p, int layout, int ns, int det, cudaStream_t st) {
  return p.v[0][0].rs ? launch_batch_phys<ST, true>(p, layout, ns, det, st)
                      : launch_batch_phys<ST, false>(p, layout, ns, det, st);
}

static cudaError_t launch_batch(const BatchLaunch &p, int storage, int layout, int ns, int det, cudaStream_t st) {
  switch (storage) {
    case LBM_FP32: return launch_batch_modes<LBM_FP32>(p, layout, ns, det, st);
    case LBM_FP16_DEV: return launch_batch_modes<LBM_FP16_DEV>(p, layout, ns, det, st);
    default: return launch_batch_modes<LBM_BF16_DEV>(p, layout, ns, det, st);
  }
}

template <int ST, bool RS>
static cudaError_t launch_batch_split_phys(const BatchLaunch &p, int layout, int ns, int det, cudaStream_t st) {
  switch (p.v[0][0].phys) {
    case kPhysBary: return launch_batch_split_st<ST, RS, kPhysBary>(p, layout, ns, det, st);
    case kPhysChannel: return launch_batch_split_st<ST, RS, kPhysChannel>(p, layout, ns, det, st);
    default: return launch_batch_split_st<ST, RS, kPhysCarrier>(p, layout, ns, det, st);
  }
}

static cudaError_t launch_batch_split(const BatchLaunch &p, int storage, int layout, int ns, int det,
                                      cudaStream_t st) {
  const bool rs = p.v[0][0].rs != 0;
  switch (storage) {
    case LBM_FP32:
      return rs ? launch_batch_split_phys<LBM_FP32, true>(p, layout, ns, det, st)
                : launch_batch_split_phys<LBM_FP32, false>(p, layout, ns, det, st);
    case LBM_FP16_DEV:
      return rs ? launch_batch_split_phys<LBM_FP16_DEV, true>(p, layout, ns, det, st)
                : launch_batch_split_phys<LBM_FP16_DEV, false>(p, layout, ns, det, st);
    default:
      return rs ? launch_batch_split_phys<LBM_BF16_DEV, true>(p, layout, ns, det, st)
                : launch_batch_split_phys<LBM_BF16_DEV, false>(p, layout, ns, det, st);
  }
}

cudaError_t launch_plane_sums(const ObsArgs &o, int storage, int layout, int ns, cudaStream_t st) {
  switch (storage) {
    case LBM_FP32: return launch_plane_sums_st<LBM_FP32>(o, layout, ns, st);
    case LBM_FP16_DEV: return launch_plane_sums_st<LBM_FP16_DEV>(o, layout, ns, st);
    default: return launch_plane_sums_st<LBM_BF16_DEV>(o, layout, ns, st);
  }
}

cudaError_t launch_export(const StepArgs &a, int parity, int storage, int layout, int ns, int which, float *dst,
                          cudaStream_t st) {
  switch (storage) {
    case LBM_FP32: return launch_export_st<LBM_FP32>(a, parity, layout, ns, which, dst, st);
    case LBM_FP16_DEV: return launch_export_st<LBM_FP16_DEV>(a, parity, layout, ns, which, dst, st);
    default: return launch_export_st<LBM_BF16_DEV>(a, parity, layout, ns, which, dst, st);
  }
}

__global__ void sum_columns_kernel(const double *in, int64_t rows, int cols, double *out) {
  const int col = blockIdx.x;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += in[r * cols + col];
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[col] = sh[0];
}

cudaError_t launch_sum_columns(const double *in, int64_t rows, int cols, double *out, cudaStream_t st) {
  sum_columns_kernel<<<cols, 256, 0, st>>>(in, rows, cols, out);
  return cudaGetLastError();
}

// reactant wall hits of the last step per node (summed over the node's link
// slots node_off[k] .. node_off[k + 1] - 1 under the random sputtering
// matrix; node_off null: one slot per node)
template <bool DET>
__global__ void site_map_kernel(const void *A, int64_t n, const int32_t *node_off, float coef, float *dst) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  float h = 0.f;
  if (!node_off)
    h = acc_get<DET>(A, k);
  else
    for (int32_t l = node_off[k]; l < node_off[k + 1]; ++l) h += acc_get<DET>(A, l);
  dst[k] = coef * h;
}

cudaError_t launch_site_map(const void *A_prev_R, int det, int64_t n_nodes, const int32_t *node_off, float coef,
                            float *dst, cudaStream_t st) {
  if (n_nodes == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n_nodes + 255) / 256);
  if (det)
    site_map_kernel<true><<<grid, 256, 0, st>>>(A_prev_R, n_nodes, node_off, coef, dst);
  else
    site_map_kernel<false><<<grid, 256, 0, st>>>(A_prev_R, n_nodes, node_off, coef, dst);
  return cudaGetLastError();
}

static StepArgs make_args_at(const lbm_sim *s, int64_t t);

StepArgs make_args(const lbm_sim *s) { return make_args_at(s, s->t); }

#ifdef LBM_CHECKED
// The bounds-check record of the checked build: one device word per process,
// allocated on first use and kept for the process's life.
static unsigned long long *check_word() {
  static unsigned long long *w = nullptr;
  if (!w && cudaMalloc(&w, sizeof(*w)) == cudaSuccess) cudaMemset(w, 0, sizeof(*w));
  return w;
}
#endif

// Kernel arguments for the step that advances the simulation from time t.
static StepArgs make_args_at(const lbm_sim *s, const int64_t t) {
  const lbm_geometry *g = s->g;
  StepArgs a{};
  a.f = s->f;
  a.fs = static_cast<char *>(s->f) + carrier_bytes(s->n_pad, s->storage);
  a.n_pad = s->n_pad;
  a.n_lat = s->n_lat;
  a.n_nodes = g->n_nodes;
  a.nx = g->nx;
  a.ny = g->ny;
  a.nz = g->nz;
  {
    const FastDiv dp = fast_div_of((uint32_t)(g->nx * g->ny)), dx = fast_div_of((uint32_t)g->nx);
    a.div_plane_m = dp.m;
    a.div_nx_m = dx.m;
    a.div_sh = dp.s1 | (dp.s2 << 8) | (dx.s1 << 16) | (dx.s2 << 24);
  }
  a.periodic_z = g->bc == LBM_BC_PERIODIC;
  a.mask = g->mask;
  a.idx = g->idx;
  const bool dense = s->layout == LBM_LAYOUT_DENSE;
  a.nbm = dense ? g->nbm_dense : g->nbm_fluid;
  a.fcell = g->fcell;
  a.inv_b = g->inv_b;
  a.node_cell = g->node_cell;
  // ring of three [2][acc_row] buffers of the accumulator's type
  const size_t ring = 2 * (size_t)s->acc_row * (s->det ? sizeof(acc_t) : sizeof(float));
  char *A = static_cast<char *>(s->A);
  a.A_prev = A + ((t + 2) % 3) * ring;  // buffer of step t-1
  a.A_cur = A + (t % 3) * ring;
  a.A_next = A + ((t + 1) % 3) * ring;
  a.det = s->det;
  const int64_t ubsz = 2 * 5 * g->plane;
  a.ub_prev = s->ub + ((t + 1) & 1) * ubsz;
  a.ub_cur = s->ub + (t & 1) * ubsz;
  a.node_cum = s->node_cum;
  a.flux_cum = s->flux_cum;
  a.n_lo_warps = s->n_lo_warps;
  a.hi_warp = s->hi_warp;
  a.n_lat_warps = s->n_lat_warps;
  a.fast_list = s->wlist;
  a.gen_list = s->wlist ? s->wlist + s->n_fast + s->n_wall : nullptr;
  a.n_fast = s->n_fast;
  a.n_wall = s->n_wall;
  a.n_uni = s->n_uni;
  a.n_gen = s->n_gen;
  a.omega = (float)(1.0 / s->prm.tau);
  a.c_in = (float)s->prm.c_in;
  a.drho_in = (float)(s->prm.rho_in - 1.0);
  a.drho_out = (float)(s->prm.rho_out - 1.0);
  a.em_R = (float)(1.0 - (s->prm.desorb ? s->p * s->prm.pS_R : s->prm.pS_R));
  a.em_PR = (float)(s->p * s->prm.pS_R);
  a.em_P = (float)(1.0 - s->prm.pS_P);
  a.parity = (int32_t)(t & 1);
  // distinct per simulation (geometry seed) and step
  a.seed_mix = seed_mix_of(g->seed);
  a.t = t;
  a.acc_row = s->acc_row;
  a.node_off = s->node_off;
  a.rs = s->rs;
  a.bary = s->bary;
  a.vel_in = s->vel_in;
  a.u_in = (float)s->prm.u_in;
  a.omega_s = (float)(1.0 / (s->prm.tau_s > 0.0 ? s->prm.tau_s : s->prm.tau));
  a.g_z = (float)s->prm.g_z;
  a.phys = s->phys;
  a.sp_bb = s->sp_bb;
#ifdef LBM_CHECKED
  a.check = check_word();
#endif
  a.halo_lo = g->halo_lo;
  a.halo_hi = g->halo_hi;
  a.hash_base = dense ? (uint32_t)((int64_t)g->z_base * g->plane) : (uint32_t)g->fluid_base;
  a.bank_lo = (int32_t)(g->halo_lo ? g->node_plane_h[2] : 0);
  a.bank_hi = (int32_t)(g->halo_hi ? g->node_plane_h[g->nz - 2] : g->n_nodes);
  a.rs_key = splitmix64_next(s->prm.sputter_seed);
  a.cell_bits = g->nbm_dense;
  return a;
}

static int run_plane_sums(lbm_sim *s, std::vector<double> &ps) {
  ObsArgs o{};
  o.s = make_args(s);
  o.parity = (int)(s->t & 1);
  o.lat_plane = s->layout == LBM_LAYOUT_DENSE ? s->g->cell_plane_d : s->g->fl_plane_d;
  o.node_plane = s->g->node_plane_d;
  o.plane_sums = s->plane_sums;
  cudaStream_t st = s->mem.stream;
  LBM_CUDA_TRY(launch_plane_sums(o, s->storage, s->layout, s->ns, st), "plane sums");
  ps.resize(kPlaneCols * (size_t)s->g->nz);
  LBM_CUDA_TRY(cudaMemcpyAsync(ps.data(), s->plane_sums, sizeof(double) * ps.size(), cudaMemcpyDeviceToHost, st),
               "copy plane sums");
  return LBM_OK;
}

// Per lattice warp: 0 when no entry is live (padding, or all solid in dense
// addressing), 1 when every live entry is plain, 3 when every live entry is
// on a fast plane and some touch a solid (a wall warp), 2 otherwise. Fluid-only
// addressing also gives, per plain warp of 32 live entries, the shift
// D = cell - entry when it is one value for the whole warp and every
// neighbour cell c + c_k of every entry has the entry c + c_k - D (then the
// odd step needs neither fcell nor idx), else INT32_MIN.
template <int LAYOUT>
__global__ void warp_class_kernel(const StepArgs a, uint8_t *cls, int32_t *shift) {
  const int64_t L64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t L = (int32_t)L64;
  bool live = L64 < a.n_lat;
  bool plain = true, onplane = true, halo = false;
  if (live) {
    const int32_t cell = (LAYOUT == LBM_LAYOUT_DENSE) ? L : a.fcell[L];
    if (LAYOUT == LBM_LAYOUT_DENSE && a.mask[cell]) live = false;
    halo = live && halo_plane(a, cell / (a.nx * a.ny));
    live = live && !halo;
    if (live) {
      plain = fast_entry(a, cell, a.nbm[L]);
      onplane = fast_plane(a, cell);
    }
  }
  // a warp holding a halo cell (not stepped) and live ones takes the general path
  const unsigned any_live = __ballot_sync(0xffffffffu, live);
  const unsigned all_plain = __all_sync(0xffffffffu, plain && !halo);
  const unsigned all_onplane = __all_sync(0xffffffffu, onplane && !halo);
  if ((threadIdx.x & 31) == 0 && (L64 >> 5) < a.n_lat_warps)
    cls[L64 >> 5] = !any_live ? 0 : (all_plain ? 1 : (all_onplane ? 3 : 2));
  if (LAYOUT == LBM_LAYOUT_FLUID) {
    // (a plain entry lies on a fast plane, so its neighbours are in the box
    // and all fluid: idx holds their entries)
    bool same = live && plain;
    int32_t D = 0;
    if (same) {
      const int32_t cell = a.fcell[L];
      D = cell - L;
      const int32_t plane = a.nx * a.ny;
      const int z = cell / plane;
      const int32_t xy = cell - z * plane;
      const int y = xy / a.nx;
      const Nbr nb(cell, xy - y * a.nx, y, z, a.nx, a.ny, a.nz, a.periodic_z);
      for (int k = 1; k < kQ; ++k) {
        const int32_t c2 = nb.at(cx(k), cy(k), cz(k));
        if (a.idx[c2] != c2 - D) same = false;
      }
    }
    const int32_t D0 = __shfl_sync(0xffffffffu, D, 0);
    const unsigned all_same = __all_sync(0xffffffffu, same && D == D0);
    if ((threadIdx.x & 31) == 0 && (L64 >> 5) < a.n_lat_warps) shift[L64 >> 5] = all_same ? D0 : INT32_MIN;
  }
}

cudaError_t launch_warp_class(const StepArgs &a, int layout, uint8_t *cls, int32_t *shift, cudaStream_t st) {
  const unsigned grid = (unsigned)(((int64_t)a.n_lat_warps * 32 + 255) / 256);
  if (grid == 0) return cudaSuccess;
  if (layout == LBM_LAYOUT_DENSE)
    warp_class_kernel<LBM_LAYOUT_DENSE><<<grid, 256, 0, st>>>(a, cls, shift);
  else
    warp_class_kernel<LBM_LAYOUT_FLUID><<<grid, 256, 0, st>>>(a, cls, shift);
  return cudaGetLastError();
}

// The warp lists of a simulation, from the per-warp classes: the fast
// kernel's warps, then the general warps (increasing). The fast list begins
// with the region warps (fluid-only addressing: plain warps numbered in cell
// order up to one shift that their neighbours share; each carries the number
// of its shift, one per distinct shift, the first kUniRegions met in warp
// order), then the other plain and the wall warps together in increasing
// order, a wall warp marked by the sign bit. In increasing order the wall
// warps of a plane follow its plain warps, so the odd step's gathers of a
// wall warp find its plain neighbours' lines still in L2. The shifts follow
// the lists at word n_lat_warps.
static cudaError_t build_warp_lists(lbm_sim *s, cudaStream_t st) {
  const int64_t nw = s->n_lat_warps;
  if (nw == 0) return cudaSuccess;
  const bool fluid = s->layout == LBM_LAYOUT_FLUID;
  uint8_t *dcls = (uint8_t *)s->mem.alloc((size_t)nw);
  int32_t *dshift = fluid ? (int32_t *)s->mem.alloc(sizeof(int32_t) * (size_t)nw) : nullptr;
  if (!dcls || (fluid && !dshift)) {
    if (dcls) s->mem.free(dcls, (size_t)nw);
    if (dshift) s->mem.free(dshift, sizeof(int32_t) * (size_t)nw);
    return cudaErrorMemoryAllocation;
  }
  StepArgs a = make_args(s);
  std::vector<uint8_t> cls((size_t)nw);
  std::vector<int32_t> shift(fluid ? (size_t)nw : 0);
  cudaError_t e = launch_warp_class(a, s->layout, dcls, dshift, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cls.data(), dcls, (size_t)nw, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && fluid)
    e = cudaMemcpyAsync(shift.data(), dshift, sizeof(int32_t) * (size_t)nw, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  s->mem.free(dcls, (size_t)nw);
  if (dshift) s->mem.free(dshift, sizeof(int32_t) * (size_t)nw);
  if (e != cudaSuccess) return e;
  std::vector<int32_t> lst;
  lst.reserve((size_t)nw + kUniTable);
  std::vector<int32_t> table(kUniTable, 0);  // table[r]: the shift of region r (word 0 unused)
  std::vector<uint8_t> in_region((size_t)nw, 0);
  int n_regions = 0, last = 0;
  s->n_fast = s->n_wall = s->n_uni = 0;
  if (fluid) {
    for (int64_t w = 0; w < nw; ++w) {
      if (cls[(size_t)w] != 1 || shift[(size_t)w] == INT32_MIN) continue;
      const int32_t D = shift[(size_t)w];
      int r = (last > 0 && table[last] == D) ? last : 0;
      for (int q = 1; q <= n_regions && r == 0; ++q)
        if (table[q] == D) r = q;
      if (r == 0 && n_regions < kUniRegions) table[r = ++n_regions] = D;
      if (r == 0) continue;
      last = r;
      in_region[(size_t)w] = 1;
      lst.push_back((int32_t)((uint32_t)w | ((uint32_t)r << kUniShift)));
      ++s->n_uni;
      ++s->n_fast;
    }
  }
  for (int64_t w = 0; w < nw; ++w) {
    if (cls[(size_t)w] == 1 && !in_region[(size_t)w]) {
      lst.push_back((int32_t)w);
      ++s->n_fast;
    } else if (cls[(size_t)w] == 3) {
      lst.push_back((int32_t)((uint32_t)w | kWallWarp));
      ++s->n_wall;
    }
  }
  s->last_warp_cls = cls[(size_t)nw - 1];
  for (int64_t w = 0; w < nw; ++w)
    if (cls[(size_t)w] == 2) lst.push_back((int32_t)w);
  s->n_gen = (int32_t)lst.size() - s->n_fast - s->n_wall;
  lst.resize((size_t)nw, 0);
  lst.insert(lst.end(), table.begin(), table.end());
  e = cudaMemcpyAsync(s->wlist, lst.data(), sizeof(int32_t) * lst.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // lst is pageable and leaves scope
  return e;
}

}  // namespace lbm

using namespace lbm;

extern "C" {

const char *lbm_error_string(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "out of device memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_DIVERGED: return "simulation diverged (NaN or non-positive density)";
    case LBM_ERR_STATE: return "invalid state";
    case LBM_ERR_TIMEOUT: return "a bounded wait inside a kernel ran past its limit";
    default: return "unknown error";
  }
}

const char *lbm_last_error(void) { return g_last_error.c_str(); }

int lbm_create_geometry(const lbm_geometry_desc *d, void *stream, const lbm_allocator *alloc, lbm_geometry **out) {
  NvtxRange nvtx_range("lbm_create_geometry");
  if (!d || !out) return arg_fail("null argument");
  *out = nullptr;
  if (d->nx < 1 || d->ny < 1 || d->nz < 4) return arg_fail("box must be at least 1 x 1 x 4");
  const int64_t n = (int64_t)d->nx * d->ny * d->nz;
  if (n >= (int64_t)1 << 31) return arg_fail("box larger than 2^31 - 1 cells");
  if (d->bc_z != LBM_BC_PRESSURE && d->bc_z != LBM_BC_PERIODIC) return arg_fail("bc_z");
  if ((d->halo_lo != 0 && d->halo_lo != 1) || (d->halo_hi != 0 && d->halo_hi != 1)) return arg_fail("halo flags");
  if ((d->halo_lo || d->halo_hi) && (!d->mask || d->bc_z != LBM_BC_PRESSURE))
    return arg_fail("a sub-domain with halo planes needs a caller mask and LBM_BC_PRESSURE");
  if ((d->halo_lo || d->halo_hi) && d->nz < 2 * (d->halo_lo + d->halo_hi) + 1)
    return arg_fail("a sub-domain needs at least one plane of its own besides its halo planes");
  if (d->fluid_base < 0 || d->z_base < 0) return arg_fail("fluid_base / z_base");
  if (!d->mask) {
    if (d->slab_z0 < 0 || d->slab_z1 > d->nz || d->slab_z0 > d->slab_z1) return arg_fail("slab outside the box");
    if (!(d->porosity >= 0.0 && d->porosity <= 1.0)) return arg_fail("porosity outside [0, 1]");
    if (!(d->corr_len >= 0.0) || d->corr_len > 1e4) return arg_fail("corr_len");
  }
  lbm_geometry *g = new (std::nothrow) lbm_geometry();
  if (!g) return LBM_ERR_OOM;
  g->nx = d->nx;
  g->ny = d->ny;
  g->nz = d->nz;
  // chord length over the slab; a caller mask without a valid slab uses the box
  const bool slab_ok = d->slab_z0 >= 0 && d->slab_z0 < d->slab_z1 && d->slab_z1 <= d->nz;
  g->z0 = (d->mask && !slab_ok) ? 0 : d->slab_z0;
  g->z1 = (d->mask && !slab_ok) ? d->nz : d->slab_z1;
  g->bc = d->bc_z;
  g->halo_lo = d->halo_lo;
  g->halo_hi = d->halo_hi;
  g->fluid_base = d->fluid_base;
  g->z_base = d->z_base;
  g->seed = d->seed;
  g->n = n;
  g->plane = (int64_t)d->nx * d->ny;
  cudaGetDevice(&g->device);
  g->mem.stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) {
    g->mem.a = *alloc;
    g->mem.has = true;
  }
  std::vector<uint8_t> hmask((size_t)n);
  if (d->mask) {
    // copy and check in one parallel pass
    int64_t bad = 0, inert = 0;
    const uint8_t *src = d->mask;
    uint8_t *hm = hmask.data();
#pragma omp parallel for reduction(+ : bad, inert) schedule(static)
    for (int64_t c = 0; c < n; ++c) {
      const uint8_t v = src[c];
      hm[c] = v;
      bad += v > 2;
      inert += v == 2;
    }
    if (bad) {
      delete g;
      return arg_fail("mask values must be 0 (fluid), 1 (catalytic solid) or 2 (inert solid)");
    }
    g->n_inert = inert;
  } else
    grf_mask(d->nx, d->ny, d->nz, d->slab_z0, d->slab_z1, d->porosity, d->corr_len, d->seed, hmask.data());
  if (g->bc == LBM_BC_PRESSURE) {
    for (int z : {0, 1, d->nz - 2, d->nz - 1}) {
      if ((g->halo_lo && z < 2) || (g->halo_hi && z >= d->nz - 2)) continue;  // halo planes may hold solid
      for (int64_t k = 0; k < g->plane; ++k)
        if (hmask[(size_t)(z * g->plane + k)]) {
          delete g;
          return arg_fail("solid cell in an inlet/outlet plane or next to one (planes 0, 1, nz-2, nz-1)");
        }
    }
  }
  g->delta = chord_length(g->nx, g->ny, g->nz, g->z0, g->z1, hmask.data());
  // geometry identity for checkpoints: FNV-1a (64-bit) of every 1 MiB chunk of
  // the mask, in parallel, then FNV-1a of the chunk hashes in order
  constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ULL, kFnvPrime = 0x100000001b3ULL;
  constexpr int64_t kChunk = (int64_t)1 << 20;
  const int64_t n_chunks = (n + kChunk - 1) / kChunk;
  std::vector<uint64_t> chunk_hash((size_t)n_chunks);
  const uint8_t *hm = hmask.data();
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n_chunks; ++k) {
    uint64_t h = kFnvBasis;
    const int64_t end = std::min(n, (k + 1) * kChunk);
    for (int64_t c = k * kChunk; c < end; ++c) h = (h ^ hm[c]) * kFnvPrime;
    chunk_hash[(size_t)k] = h;
  }
  uint64_t hsh = kFnvBasis;
  for (uint64_t v : chunk_hash)
    for (int byte = 0; byte < 8; ++byte) hsh = (hsh ^ ((v >> (8 * byte)) & 0xffu)) * kFnvPrime;
  g->mask_hash = hsh;
  cudaStream_t st = (cudaStream_t)stream;
  g->mask = (uint8_t *)g->mem.alloc((size_t)n);
  g->idx = (int32_t *)g->mem.alloc(sizeof(int32_t) * n);
  g->b = (int32_t *)g->mem.alloc(sizeof(int32_t) * n);
  g->nbm_dense = (uint32_t *)g->mem.alloc(sizeof(uint32_t) * n);
  if (!g->mask || !g->idx || !g->b || !g->nbm_dense) {
    lbm_geometry_free(g);
    set_error("geometry allocation failed");
    return LBM_ERR_OOM;
  }
  cudaError_t e = cudaMemcpyAsync(g->mask, hmask.data(), (size_t)n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // hmask is pageable and leaves scope
  if (e == cudaSuccess) e = build_structures(g, st);
  if (e != cudaSuccess) {
    lbm_geometry_free(g);
    if (e == cudaErrorMemoryAllocation) {
      set_error("geometry allocation failed");
      return LBM_ERR_OOM;
    }
    return cuda_fail(e, "geometry build");
  }
  *out = g;
  return LBM_OK;
}

int lbm_geometry_info(const lbm_geometry *g, int64_t *n_fluid, int64_t *n_nodes, int64_t *n_links, double *delta) {
  if (!g) return arg_fail("null geometry");
  if (n_fluid) *n_fluid = g->n_fluid;
  if (n_nodes) *n_nodes = g->n_nodes;
  if (n_links) *n_links = g->n_links;
  if (delta) *delta = g->delta;
  return LBM_OK;
}

int lbm_geometry_export(const lbm_geometry *g, uint8_t *mask, int32_t *fluid_idx, int32_t *node_idx, int32_t *b,
                        int64_t *links) {
  if (!g) return arg_fail("null geometry");
  cudaStream_t st = g->mem.stream;
  const int64_t n = g->n;
  std::vector<uint8_t> m((size_t)n);
  std::vector<int32_t> idx((size_t)n);
  LBM_CUDA_TRY(cudaMemcpyAsync(m.data(), g->mask, (size_t)n, cudaMemcpyDeviceToHost, st), "export mask");
  LBM_CUDA_TRY(cudaMemcpyAsync(idx.data(), g->idx, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st), "export idx");
  if (b) LBM_CUDA_TRY(cudaMemcpyAsync(b, g->b, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st), "export b");
  std::vector<uint32_t> nbm;
  if (links) {
    nbm.resize((size_t)n);
    LBM_CUDA_TRY(cudaMemcpyAsync(nbm.data(), g->nbm_dense, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, st),
                 "export nbm");
  }
  LBM_CUDA_TRY(cudaStreamSynchronize(st), "export sync");
  if (mask) std::memcpy(mask, m.data(), (size_t)n);
  // fluid cells numbered in linear order (the lattice entries of fluid-only
  // addressing are ordered differently within each plane)
  int64_t nf = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (fluid_idx) fluid_idx[c] = m[c] ? -1 : (int32_t)nf;
    nf += m[c] ? 0 : 1;
    if (node_idx) node_idx[c] = m[c] ? idx[c] : -1;
  }
  if (links) {
    int64_t k = 0;
    const int64_t plane = g->plane;
    for (int64_t c = 0; c < n; ++c) {
      if (m[c] || !nbm[c]) continue;
      const int z = (int)(c / plane), y = (int)((c % plane) / g->nx), x = (int)(c % g->nx);
      for (int i = 1; i < kQ; ++i) {
        if (!((nbm[c] >> i) & 1u)) continue;
        const int xx = (x + cx(i) + g->nx) % g->nx, yy = (y + cy(i) + g->ny) % g->ny;
        const int zz = ((z + cz(i)) % g->nz + g->nz) % g->nz;
        const int64_t t = ((int64_t)zz * g->ny + yy) * g->nx + xx;
        if (m[t] != 1) continue;  // inert solid: a bounce-back link, not a catalytic one
        links[3 * k + 0] = c;
        links[3 * k + 1] = i;
        links[3 * k + 2] = t;
        ++k;
      }
    }
  }
  return LBM_OK;
}

void lbm_geometry_free(lbm_geometry *g) {
  if (!g) return;
  DevAlloc &m = g->mem;
  m.free(g->mask, g->n);
  m.free(g->idx, sizeof(int32_t) * g->n);
  m.free(g->b, sizeof(int32_t) * g->n);
  m.free(g->nbm_dense, sizeof(uint32_t) * g->n);
  m.free(g->nbm_fluid, sizeof(uint32_t) * std::max<int64_t>(g->n_fluid, 1));
  m.free(g->fcell, sizeof(int32_t) * std::max<int64_t>(g->n_fluid, 1));
  m.free(g->inv_b, sizeof(float) * std::max<int64_t>(g->n_nodes, 1));
  m.free(g->node_cell, sizeof(int32_t) * std::max<int64_t>(g->n_nodes, 1));
  m.free(g->fl_plane_d, sizeof(int64_t) * (g->nz + 1));
  m.free(g->node_plane_d, sizeof(int64_t) * (g->nz + 1));
  m.free(g->cell_plane_d, sizeof(int64_t) * (g->nz + 1));
  cudaStreamSynchronize(m.stream);
  delete[] g->fl_plane_h;
  delete[] g->node_plane_h;
  delete g;
}

// LBM_LAYOUT_AUTO: fluid-only addressing below a fluid fraction of 0.98.
// Measured on GB300 (192x192x384, C+R+P, FP32 and FP16), fluid-only was as
// fast as dense or faster at every fluid fraction from 0.50 to 0.98 (equal
// at 0.98 in FP32); dense keeps boxes that are (almost) all fluid free of
// the indirection.
static int resolve_layout(const lbm_geometry *g, int layout) {
  if (layout == LBM_LAYOUT_DENSE || layout == LBM_LAYOUT_FLUID) return layout;
  const double fluid_frac = (double)g->n_fluid / (double)g->n;
  return fluid_frac < 0.98 ? LBM_LAYOUT_FLUID : LBM_LAYOUT_DENSE;
}

static int check_params(const lbm_params *p) {
  if (!p) return arg_fail("null params");
  if (!(p->tau > 0.5)) return arg_fail("tau must exceed 0.5");
  if (p->n_species != 1 && p->n_species != 2) return arg_fail("n_species must be 1 or 2");
  if (p->storage != LBM_FP32 && p->storage != LBM_FP16_DEV && p->storage != LBM_BF16_DEV) return arg_fail("storage");
  if (p->layout < LBM_LAYOUT_AUTO || p->layout > LBM_LAYOUT_FLUID) return arg_fail("layout");
  if (!(p->pS_R >= 0 && p->pS_R <= 1 && p->pS_P >= 0 && p->pS_P <= 1)) return arg_fail("sticking probabilities");
  if (!(p->rho_in > 0 && p->rho_out > 0 && p->c_in >= 0)) return arg_fail("densities");
  if (!(p->c_init >= 0.0 && p->c_init <= 4.0)) return arg_fail("c_init must lie in [0, 4]");
  if (p->sputter != LBM_S_UNIFORM && p->sputter != LBM_S_RANDOM && p->sputter != LBM_S_BOUNCEBACK)
    return arg_fail("sputter");
  if (p->desorb != 0 && p->desorb != 1) return arg_fail("desorb");
  if (p->sputter == LBM_S_BOUNCEBACK && p->velocity != LBM_U_CARRIER)
    return arg_fail("species bounce-back needs the carrier velocity");
  if (p->velocity != LBM_U_CARRIER && p->velocity != LBM_U_BARYCENTRIC) return arg_fail("velocity");
  if (p->inlet != LBM_INLET_PRESSURE && p->inlet != LBM_INLET_VELOCITY) return arg_fail("inlet");
  if (p->inlet == LBM_INLET_VELOCITY && !(std::fabs(p->u_in) <= 0.3)) return arg_fail("u_in must lie in [-0.3, 0.3]");
  if (!(p->tau_s == 0.0 || p->tau_s > 0.5)) return arg_fail("tau_s must be 0 (the carrier's tau) or exceed 0.5");
  if (!(std::fabs(p->g_z) <= 1e-2)) return arg_fail("g_z must lie in [-0.01, 0.01]");
  if (p->g_z != 0.0 && p->velocity != LBM_U_CARRIER) return arg_fail("a body force needs the carrier velocity");
  // a forced flow gains ~(1 - omega/2) 3 g per step in each carrier deviation,
  // below the binary16 / bfloat16 resolution of deviations of order 3 u
  if (p->g_z != 0.0 && p->storage != LBM_FP32) return arg_fail("a body force needs LBM_FP32 storage");
  return LBM_OK;
}

static void sim_sizes(const lbm_geometry *g, const lbm_params *p, int layout, lbm_sim *s) {
  s->n_lat = layout == LBM_LAYOUT_DENSE ? g->n : g->n_fluid;
  s->n_pad = pad64(std::max<int64_t>(s->n_lat, 1));
  s->n_nodes_pad = pad64(std::max<int64_t>(g->n_nodes, 1));
  s->rs = p->sputter == LBM_S_RANDOM ? 1 : 0;
  s->bary = p->velocity == LBM_U_BARYCENTRIC ? 1 : 0;
  // the kernel variant: the channel one only where a channel ingredient is in use
  s->sp_bb = p->sputter == LBM_S_BOUNCEBACK ? 1 : 0;
  const bool channel =
      g->n_inert > 0 || p->g_z != 0.0 || (p->tau_s > 0.0 && p->tau_s != p->tau) || s->sp_bb;
  s->phys = s->bary ? kPhysBary : (channel ? kPhysChannel : kPhysCarrier);
  s->vel_in = p->inlet == LBM_INLET_VELOCITY ? 1 : 0;
  s->acc_row = s->rs ? pad64(std::max<int64_t>(g->n_links, 1)) : s->n_nodes_pad;
  s->ns = 1 + p->n_species;
  const int64_t work = std::max(s->n_lat, g->n_nodes);
  s->n_blocks = std::max<int64_t>((work + kBlock - 1) / kBlock, 1);
  s->n_lat_warps = (int32_t)((s->n_lat + 31) / 32);
  // face flows: one slot per lattice warp overlapping planes 0, 1 or nz-2, nz-1
  int64_t lo_end = 0, hi_start = 0;
  if (layout == LBM_LAYOUT_DENSE) {
    lo_end = 2 * g->plane;
    hi_start = (int64_t)(g->nz - 2) * g->plane;
  } else {
    lo_end = g->fl_plane_h[2];
    hi_start = g->fl_plane_h[g->nz - 2];
  }
  // (a halo end has no inlet/outlet face and no slots)
  s->n_lo_warps = g->halo_lo ? 0 : (int32_t)((lo_end + 31) / 32);
  s->hi_warp = g->halo_hi ? s->n_lat_warps : (int32_t)std::max<int64_t>(hi_start / 32, s->n_lo_warps);
  s->n_flux_slots = s->n_lo_warps + std::max<int64_t>(s->n_lat_warps - s->hi_warp, 0);
}

static size_t sim_bytes(const lbm_geometry *g, const lbm_sim *s, int storage) {
  size_t b = 0;
  b += (size_t)s->ns * kQ * s->n_pad * storage_bytes(storage);
  b += sizeof(acc_t) * 3 * 2 * s->acc_row;
  if (s->rs) b += sizeof(int32_t) * (g->n_nodes + 1);
  b += sizeof(float) * 2 * 2 * 5 * g->plane;
  b += sizeof(double) * 2 * s->n_blocks;
  b += sizeof(double) * 6 * std::max<int64_t>(s->n_flux_slots, 1);
  b += sizeof(double) * kPlaneCols * g->nz + sizeof(double) * 8;
  b += sizeof(int32_t) * (std::max<int64_t>(s->n_lat_warps, 1) + kUniTable);  // warp lists, region shifts
  b += sizeof(BatchSync);  // step counters of a single-launch batch led by this simulation
  return b;
}

int lbm_footprint(const lbm_geometry *g, const lbm_params *prm, size_t *bytes) {
  if (!g || !bytes) return arg_fail("null argument");
  int rc = check_params(prm);
  if (rc) return rc;
  lbm_sim tmp;
  sim_sizes(g, prm, resolve_layout(g, prm->layout), &tmp);
  *bytes = sim_bytes(g, &tmp, prm->storage);
  return LBM_OK;
}

int lbm_request_footprint(const lbm_geometry_desc *d, const lbm_params *prm, size_t *bytes) {
  if (!d || !bytes) return arg_fail("null argument");
  int rc = check_params(prm);
  if (rc) return rc;
  if (d->nx < 1 || d->ny < 1 || d->nz < 4) return arg_fail("box must be at least 1 x 1 x 4");
  const int64_t n = (int64_t)d->nx * d->ny * d->nz;
  // geometry: mask, idx, b, dense neighbour masks per cell; fluid-entry
  // arrays and node arrays (inv_b, node_cell) bounded by the cell count;
  // plane tables
  size_t geo = (size_t)n * (1 + 4 + 4 + 4) + (size_t)n * (4 + 4) + (size_t)n * (4 + 4) + 3 * sizeof(int64_t) * (d->nz + 1);
  // simulation with every cell a lattice entry and a node (the upper bound)
  lbm_geometry g;
  g.nx = d->nx;
  g.ny = d->ny;
  g.nz = d->nz;
  g.n = n;
  g.plane = (int64_t)d->nx * d->ny;
  g.n_fluid = n;
  g.n_nodes = n;
  g.n_links = 9 * n;  // links join a fluid cell and a node: at most 18 min(n_fluid, n_nodes) <= 9 n
  std::vector<int64_t> fl(d->nz + 1);
  for (int z = 0; z <= d->nz; ++z) fl[z] = (int64_t)z * g.plane;
  g.fl_plane_h = fl.data();
  lbm_sim tmp;
  sim_sizes(&g, prm, LBM_LAYOUT_DENSE, &tmp);
  *bytes = geo + sim_bytes(&g, &tmp, prm->storage);
  g.fl_plane_h = nullptr;
  return LBM_OK;
}

static void sim_free_all(lbm_sim *s) {
  DevAlloc &m = s->mem;
  m.free(s->f, (size_t)s->ns * kQ * s->n_pad * storage_bytes(s->storage));
  m.free(s->A, sizeof(acc_t) * 3 * 2 * s->acc_row);
  m.free(s->node_off, sizeof(int32_t) * (s->g->n_nodes + 1));
  m.free(s->ub, sizeof(float) * 2 * 2 * 5 * s->g->plane);
  m.free(s->node_cum, sizeof(double) * 2 * s->n_blocks);
  m.free(s->flux_cum, sizeof(double) * 6 * std::max<int64_t>(s->n_flux_slots, 1));
  m.free(s->plane_sums, sizeof(double) * kPlaneCols * s->g->nz);
  m.free(s->red_out, sizeof(double) * 8);
  m.free(s->wlist, sizeof(int32_t) * (std::max<int64_t>(s->n_lat_warps, 1) + kUniTable));
}


// carrier at rest with density 1 + drho: d_i = drho; species 0. Every
// element of both arrays, padding included: the first n_carrier elements
// (of the storage type) are the carrier array, the rest the species array.
// The reactant (every species element with NS = 2, the low element of each
// pair with NS = 3) starts at c_sp, its initial density in the stored units.
// Initial populations, 16 bytes per thread (8 16-bit or 4 FP32 values; the
// array lengths are multiples of 64 elements and the arrays 256-byte
// aligned, so no vector straddles the carrier/species boundary or the end).
__global__ void init_pops_kernel(void *fv, int storage, int ns, int64_t n_carrier, int64_t n_elem, float drho,
                                 float c_sp) {
  const int per = storage == LBM_FP32 ? 4 : 8;
  const int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * per;
  if (k0 >= n_elem) return;
  // scaled deviation d = (f - w rho_ref) / w: the carrier's drho; the
  // species' c (R at even elements of the C+R+P pairs, P zero)
  float d[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t k = k0 + j;
    d[j] = k < n_carrier ? drho : ((ns == 2 || ((k - n_carrier) & 1) == 0) ? c_sp : 0.0f);
  }
  if (storage == LBM_FP32) {
    reinterpret_cast<float4 *>(fv)[k0 / 4] = make_float4(d[0], d[1], d[2], d[3]);
  } else {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint16_t lo, hi;
      if (storage == LBM_FP16_DEV) {
        lo = __half_as_ushort(__float2half_rn(d[2 * j]));
        hi = __half_as_ushort(__float2half_rn(d[2 * j + 1]));
      } else {
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(d[2 * j]));
        hi = __bfloat16_as_ushort(__float2bfloat16_rn(d[2 * j + 1]));
      }
      w[j] = (uint32_t)lo | ((uint32_t)hi << 16);
    }
    reinterpret_cast<uint4 *>(fv)[k0 / 8] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

int lbm_init(const lbm_geometry *g, const lbm_params *prm, void *stream, const lbm_allocator *alloc, lbm_sim **out) {
  NvtxRange nvtx_range("lbm_init");
  if (!g || !out) return arg_fail("null argument");
  *out = nullptr;
  int rc = check_params(prm);
  if (rc) return rc;
  if (prm->inlet == LBM_INLET_VELOCITY && g->bc == LBM_BC_PERIODIC)
    return arg_fail("a velocity inlet needs open z boundaries (LBM_BC_PRESSURE)");
  if (prm->velocity == LBM_U_BARYCENTRIC && g->n_inert > 0)
    return arg_fail("inert solid needs the carrier velocity");
  lbm_sim *s = new (std::nothrow) lbm_sim();
  if (!s) return LBM_ERR_OOM;
  s->g = g;
  s->prm = *prm;
  s->storage = prm->storage;
  s->layout = resolve_layout(g, prm->layout);
  // odd steps in fluid-only addressing use 32-bit element offsets between an
  // entry and its neighbours (in the same or an adjacent plane: fewer than two
  // planes of entries apart)
  if (s->layout == LBM_LAYOUT_FLUID && (2 * (int64_t)g->plane + 64) * kQ >= ((int64_t)1 << 31)) {
    delete s;
    return arg_fail("x-y plane too large for fluid-only addressing; use LBM_LAYOUT_DENSE");
  }
  s->det = prm->deterministic ? 1 : 0;
  if (prm->p_override >= 0.0 && prm->p_override <= 1.0) {
    s->p = prm->p_override;
  } else {
    const double cs = std::sqrt(1.0 / 3.0);
    s->p = (prm->Da > 0.0 && g->delta > 0.0) ? std::fmin(1.0, cs / (prm->Da * g->delta)) : 1.0;
  }
  s->mem.stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) {
    s->mem.a = *alloc;
    s->mem.has = true;
  }
  sim_sizes(g, prm, s->layout, s);
  s->bytes = sim_bytes(g, s, s->storage);
  DevAlloc &m = s->mem;
  s->f = m.alloc((size_t)s->ns * kQ * s->n_pad * storage_bytes(s->storage));
  s->A = m.alloc(sizeof(acc_t) * 3 * 2 * s->acc_row);
  s->ub = (float *)m.alloc(sizeof(float) * 2 * 2 * 5 * g->plane);
  s->node_cum = (double *)m.alloc(sizeof(double) * 2 * s->n_blocks);
  s->flux_cum = (double *)m.alloc(sizeof(double) * 6 * std::max<int64_t>(s->n_flux_slots, 1));
  s->plane_sums = (double *)m.alloc(sizeof(double) * kPlaneCols * g->nz);
  s->red_out = (double *)m.alloc(sizeof(double) * 8);
  if (s->rs) s->node_off = (int32_t *)m.alloc(sizeof(int32_t) * (g->n_nodes + 1));
  s->wlist = (int32_t *)m.alloc(sizeof(int32_t) * (std::max<int64_t>(s->n_lat_warps, 1) + kUniTable));
  if (!s->f || !s->A || !s->ub || !s->node_cum || !s->flux_cum || !s->plane_sums || !s->red_out ||
      (s->rs && !s->node_off) || !s->wlist) {
    sim_free_all(s);
    delete s;
    set_error("simulation allocation failed");
    return LBM_ERR_OOM;
  }
  cudaStream_t st = s->mem.stream;
  cudaError_t e = cudaSuccess;
  if (s->rs) {
    // link slots of the random matrix: node k owns b(k) consecutive slots
    // from node_off[k] (b from the geometry's 1/b, exact for b <= 18)
    std::vector<float> ib((size_t)g->n_nodes);
    std::vector<int32_t> off((size_t)g->n_nodes + 1, 0);
    if (g->n_nodes > 0)
      e = cudaMemcpyAsync(ib.data(), g->inv_b, sizeof(float) * g->n_nodes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int64_t k = 0; k < g->n_nodes && e == cudaSuccess; ++k)
      off[k + 1] = off[k] + (int32_t)std::lround(1.0 / (double)ib[k]);
    if (e == cudaSuccess && off[g->n_nodes] != g->n_links) e = cudaErrorInvalidValue;  // the links, counted twice
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->node_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // off is pageable and leaves scope
  }
  if (e == cudaSuccess) e = build_warp_lists(s, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->A, 0, sizeof(acc_t) * 3 * 2 * s->acc_row, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->ub, 0, sizeof(float) * 2 * 2 * 5 * g->plane, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->node_cum, 0, sizeof(double) * 2 * s->n_blocks, st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(s->flux_cum, 0, sizeof(double) * 6 * std::max<int64_t>(s->n_flux_slots, 1), st);
  if (e == cudaSuccess) {
    const int64_t n_elem = (int64_t)s->ns * kQ * s->n_pad;
    const double c_scale = s->storage == LBM_FP16_DEV ? 16384.0 : 1.0;  // the FP16 species scaling, 2^14
    const int64_t n_vec = n_elem / (s->storage == LBM_FP32 ? 4 : 8);
    init_pops_kernel<<<(unsigned)((n_vec + 255) / 256), 256, 0, st>>>(
        s->f, s->storage, s->ns, (int64_t)kQ * s->n_pad, n_elem, (float)(prm->rho_out - 1.0),
        (float)(prm->c_init * c_scale));
    e = cudaGetLastError();
  }
  std::vector<double> ps;
  if (e == cudaSuccess) {
    int r = run_plane_sums(s, ps);
    if (r) {
      sim_free_all(s);
      delete s;
      return r;
    }
    e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    sim_free_all(s);
    delete s;
    if (e == cudaErrorMemoryAllocation) {
      set_error("simulation allocation failed (warp-list scratch)");
      return LBM_ERR_OOM;
    }
    return cuda_fail(e, "init");
  }
  const bool per = g->bc == LBM_BC_PERIODIC;
  for (int z = 0; z < g->nz; ++z) {
    if (!per && (z == 0 || z == g->nz - 1)) continue;
    for (int k = 0; k < 3; ++k) s->M0[k] += ps[kPlaneCols * z + k];
  }
  *out = s;
  return LBM_OK;
}

int lbm_step(lbm_sim *s, int64_t nsteps) {
  NvtxRange nvtx_range("lbm_step");
  if (!s) return arg_fail("null simulation");
  if (nsteps < 0) return arg_fail("nsteps < 0");
  cudaStream_t st = s->mem.stream;
  for (int64_t k = 0; k < nsteps; ++k) {
    const StepArgs a = make_args(s);
    cudaError_t e = launch_step(a, s->storage, s->layout, s->ns, (int)(s->t & 1), st);
    if (e != cudaSuccess) return cuda_fail(e, "step launch");
    s->t += 1;
  }
  return LBM_OK;
}

int lbm_step_timed(lbm_sim *s, float *ms, int64_t *entries) {
  NvtxRange nvtx_range("lbm_step_timed");
  if (!s || !ms) return arg_fail("null argument");
  cudaStream_t st = s->mem.stream;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 5 && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
  if (e == cudaSuccess) {
    const StepArgs a = make_args(s);
    e = launch_step(a, s->storage, s->layout, s->ns, (int)(s->t & 1), st, ev);
    if (e == cudaSuccess) s->t += 1;
  }
  float em = 0.f, hm = 0.f;
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[4]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&em, ev[0], ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[0], ev[1], ev[2]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[1], ev[2], ev[3]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&hm, ev[3], ev[4]);
  if (e == cudaSuccess) ms[2] = em + hm;
  for (int k = 0; k < 5; ++k)
    if (ev[k]) cudaEventDestroy(ev[k]);
  if (e != cudaSuccess) return cuda_fail(e, "timed step");
  if (entries) {
    // lattice entries of each kernel's warps (the last warp may be partial)
    const int64_t last = (s->n_lat_warps > 0) ? s->n_lat - (int64_t)(s->n_lat_warps - 1) * 32 : 0;
    entries[0] = (int64_t)(s->n_fast + s->n_wall) * 32;
    entries[1] = (int64_t)s->n_gen * 32;
    if (s->last_warp_cls == 1 || s->last_warp_cls == 3) entries[0] -= 32 - last;
    else if (s->last_warp_cls == 2) entries[1] -= 32 - last;
  }
  return LBM_OK;
}

int lbm_step_batch(lbm_sim *const *sims, int n, int64_t nsteps, void *stream) {
  return lbm_step_batch_mode(sims, n, nsteps, stream, LBM_BATCH_PER_STEP);
}

int lbm_step_batch_mode(lbm_sim *const *sims, int n, int64_t nsteps, void *stream, int mode) {
  NvtxRange nvtx_range("lbm_step_batch_mode");
  if (!sims || n < 0 || nsteps < 0) return arg_fail("bad batch arguments");
  if (mode != LBM_BATCH_PER_STEP && mode != LBM_BATCH_SINGLE_LAUNCH) return arg_fail("batch mode");
  if (n == 0 || nsteps == 0) return LBM_OK;
  for (int k = 0; k < n; ++k) {
    if (!sims[k]) return arg_fail("null simulation in batch");
    for (int j = 0; j < k; ++j)
      if (sims[j] == sims[k]) return arg_fail("simulation listed twice in batch");
    if (sims[k]->g->device != sims[0]->g->device) return arg_fail("batch spans devices");
    if (sims[k]->n_blocks >= ((int64_t)1 << 31) / kMaxBatch) return arg_fail("simulation too large for a batch");
  }
  cudaStream_t st = stream ? (cudaStream_t)stream : sims[0]->mem.stream;
  // launch groups: equal (storage, layout, species, accumulation mode,
  // sputtering matrix, velocity), at most kMaxBatch simulations each
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  auto key = [&](int k) {
    return ((((sims[k]->storage * 4 + sims[k]->layout) * 4 + sims[k]->ns) * 2 + sims[k]->det) * 2 + sims[k]->rs) * 4 +
           sims[k]->phys;
  };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key(x) < key(y); });
  std::vector<std::pair<int, int>> groups;
  for (int q = 0; q < n;) {
    int r = q;
    while (r < n && key(order[r]) == key(order[q]) && r - q < kMaxBatch) ++r;
    groups.push_back({q, r});
    q = r;
  }
  // per-step launches, or several steps per launch ordered by tickets
  // (batch_step_kernel)
  int32_t max_total = 1;
  for (auto &gq : groups) {
    int64_t tot = 0;
    for (int q = gq.first; q < gq.second; ++q) tot += sims[order[q]]->n_blocks;
    max_total = std::max<int32_t>(max_total, (int32_t)tot);
  }
  const int64_t per_launch =
      mode == LBM_BATCH_PER_STEP
          ? 1
          : std::max<int64_t>(1, std::min<int64_t>(kStepsPerLaunch, (((int64_t)1 << 31) - 1) / (3 * (int64_t)max_total)));
  const size_t ng = groups.size();
  BatchSync *dsync = nullptr;
  cudaError_t e = cudaSuccess;
  // the single-launch mode's step counters: from the first simulation's
  // allocator (its lbm_footprint counts one BatchSync), on the batch stream
  DevAlloc sync_mem = sims[0]->mem;
  sync_mem.stream = st;
  if (nsteps > 1 && per_launch > 1) {
    dsync = (BatchSync *)sync_mem.alloc(sizeof(BatchSync) * ng);
    if (!dsync) {
      set_error("batch scratch allocation failed");
      return LBM_ERR_OOM;
    }
  }
  std::vector<BatchLaunch> P(ng);
  for (size_t gi = 0; gi < ng; ++gi) {
    BatchLaunch &p = P[gi];
    std::memset(&p, 0, sizeof(p));
    p.n_sims = groups[gi].second - groups[gi].first;
    int32_t total = 0, tf = 0, tg = 0, tn = 0;
    for (int q = 0; q < p.n_sims; ++q) {
      const lbm_sim *sq = sims[order[groups[gi].first + q]];
      p.block_start[q] = total;
      total += (int32_t)sq->n_blocks;
      p.fast_start[q] = tf;
      tf += (sq->n_fast + sq->n_wall + kWarpsPerBlock - 1) / kWarpsPerBlock;
      p.gen_start[q] = tg;
      tg += (sq->n_gen + kWarpsPerBlock - 1) / kWarpsPerBlock;
      p.node_start[q] = tn;
      tn += (int32_t)((sq->g->n_nodes + kBlock - 1) / kBlock);
      for (int j = 0; j < 6; ++j) p.v[q][j] = make_args_at(sq, sq->t + j);
    }
    p.block_start[p.n_sims] = total;
    p.total_blocks = total;
    p.fast_start[p.n_sims] = tf;
    p.gen_start[p.n_sims] = tg;
    p.node_start[p.n_sims] = tn;
    p.total_fast = tf;
    p.total_gen = tg;
    p.total_node = tn;
    p.sync = dsync ? dsync + gi : nullptr;
  }
  std::vector<int> flags(ng);
  bool timed_out = false;
  for (int64_t done = 0; done < nsteps && e == cudaSuccess && !timed_out;) {
    const int64_t m = dsync ? std::min<int64_t>(per_launch, nsteps - done) : 1;
    if (dsync) e = cudaMemsetAsync(dsync, 0, sizeof(BatchSync) * ng, st);
    for (size_t gi = 0; gi < ng && e == cudaSuccess; ++gi) {
      BatchLaunch &p = P[gi];
      p.k0 = (int32_t)(done % 6);  // only k0 mod 6 and t0 + k0 matter
      for (int q = 0; q < p.n_sims; ++q) p.t0[q] = sims[order[groups[gi].first + q]]->t + (done - p.k0);
      p.n_steps = (int32_t)m;
      const lbm_sim *s0 = sims[order[groups[gi].first]];
      e = (m == 1 && !dsync) ? launch_batch_split(p, s0->storage, s0->layout, s0->ns, s0->det, st)
                             : launch_batch(p, s0->storage, s0->layout, s0->ns, s0->det, st);
    }
    if (e == cudaSuccess && dsync && m > 1) {
      for (size_t gi = 0; gi < ng && e == cudaSuccess; ++gi)
        e = cudaMemcpyAsync(&flags[gi], &dsync[gi].timed_out, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // flags is pageable, dsync is reused
      for (int f : flags) timed_out = timed_out || f;
    }
    done += m;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (dsync) sync_mem.free(dsync, sizeof(BatchSync) * ng);
  if (e != cudaSuccess) return cuda_fail(e, "batched step");
  if (timed_out) {
    set_error("a step-ordering wait of the batched launch ran past its limit; the batch state is undefined");
    return LBM_ERR_TIMEOUT;
  }
  for (int q = 0; q < n; ++q) sims[q]->t += nsteps;
  return LBM_OK;
}

int lbm_observables(lbm_sim *s, lbm_obs *o) {
  NvtxRange nvtx_range("lbm_observables");
  if (!s || !o) return arg_fail("null argument");
  const lbm_geometry *g = s->g;
  cudaStream_t st = s->mem.stream;
  std::vector<double> ps;
  int r = run_plane_sums(s, ps);
  if (r) return r;
  double red[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  LBM_CUDA_TRY(launch_sum_columns(s->node_cum, s->n_blocks, 2, s->red_out, st), "sum wall hits");
  if (g->bc != LBM_BC_PERIODIC && s->n_flux_slots > 0)
    LBM_CUDA_TRY(launch_sum_columns(s->flux_cum, s->n_flux_slots, 6, s->red_out + 2, st), "sum face flows");
  else
    LBM_CUDA_TRY(cudaMemsetAsync(s->red_out + 2, 0, sizeof(double) * 6, st), "zero face flows");
  LBM_CUDA_TRY(cudaMemcpyAsync(red, s->red_out, sizeof(red), cudaMemcpyDeviceToHost, st), "copy sums");
  if (o->site_map && g->n_nodes > 0) {
    const StepArgs a = make_args(s);
    float *tmp = (float *)s->mem.alloc(sizeof(float) * g->n_nodes);
    if (!tmp) {
      set_error("site map scratch allocation failed");
      return LBM_ERR_OOM;
    }
    cudaError_t e = launch_site_map(a.A_prev, s->det, g->n_nodes, s->rs ? s->node_off : nullptr,
                                    (float)(s->p * s->prm.pS_R), tmp, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(o->site_map, tmp, sizeof(float) * g->n_nodes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    s->mem.free(tmp, sizeof(float) * g->n_nodes);
    if (e != cudaSuccess) return cuda_fail(e, "site map");
  }
  LBM_CUDA_TRY(cudaStreamSynchronize(st), "observables sync");
  const int nz = g->nz;
  const bool per = g->bc == LBM_BC_PERIODIC;
  double M[3] = {0, 0, 0}, hitsR = red[0], hitsP = red[1];
  bool bad = false;
  for (int z = 0; z < nz; ++z) {
    const double *row = &ps[(size_t)kPlaneCols * z];
    for (int k = 0; k < kPlaneCols; ++k) bad |= std::isnan(row[k]);
    if (!per && (z == 0 || z == nz - 1)) continue;
    for (int k = 0; k < 3; ++k) M[k] += row[k];
    hitsR += row[4];  // the last step's hits, not banked yet
    hitsP += row[5];
    if (o->rhoC_z) o->rhoC_z[z] = row[0];
    if (o->rhoR_z) o->rhoR_z[z] = row[1];
    if (o->rhoP_z) o->rhoP_z[z] = row[2];
    if (o->phiP_z) o->phiP_z[z] = row[3];
    if (o->react_z) o->react_z[z] = s->p * s->prm.pS_R * row[4];
  }
  if (!per) {
    for (int z : {0, nz - 1}) {
      if (o->rhoC_z) o->rhoC_z[z] = 0;
      if (o->rhoR_z) o->rhoR_z[z] = 0;
      if (o->rhoP_z) o->rhoP_z[z] = 0;
      if (o->phiP_z) o->phiP_z[z] = 0;
      if (o->react_z) o->react_z[z] = 0;
    }
  }
  const double p = s->p, pSR = s->prm.pS_R, pSP = s->prm.pS_P;
  o->step = s->t;
  o->M_C = M[0];
  o->M_R = M[1];
  o->M_P = M[2];
  const double mRin = ps[(size_t)kPlaneCols * 1 + 1], mPout = ps[(size_t)kPlaneCols * (nz - 2) + 2];
  o->eta = mRin != 0.0 ? mPout / mRin : 0.0;
  o->in_C = red[2];
  o->in_R = red[3];
  o->in_P = red[4];
  o->out_C = red[5];
  o->out_R = red[6];
  o->out_P = red[7];
  o->hits_R = hitsR;
  o->hits_P = hitsP;
  o->reacted = p * pSR * hitsR;
  o->stuck_R = s->prm.desorb ? 0.0 : pSR * (1.0 - p) * hitsR;
  o->stuck_P = pSP * hitsP;
  o->resid_C = M[0] - s->M0[0] - (o->in_C - o->out_C);
  o->resid_RP = (M[1] + M[2]) - (s->M0[1] + s->M0[2]) - (o->in_R + o->in_P - o->out_R - o->out_P) + o->stuck_R +
                o->stuck_P + (s->ns == 2 ? o->reacted : 0.0);
  o->delta = g->delta;
  o->p = p;
  o->Kn = g->delta > 0 ? std::sqrt(1.0 / 3.0) * (s->prm.tau - 0.5) / g->delta : 0.0;
  if (bad || !(M[0] > 0.0)) {
    set_error("diverged: NaN in a plane sum or non-positive carrier mass");
    return LBM_ERR_DIVERGED;
  }
  return LBM_OK;
}

static int export_common(lbm_sim *s, int which, float *dst, int dst_on_device, size_t count) {
  cudaStream_t st = s->mem.stream;
  float *out = dst;
  float *tmp = nullptr;
  if (!dst_on_device) {
    tmp = (float *)s->mem.alloc(sizeof(float) * count);
    if (!tmp) {
      set_error("export scratch allocation failed");
      return LBM_ERR_OOM;
    }
    out = tmp;
  }
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * count, st);
  const StepArgs a = make_args(s);
  if (e == cudaSuccess) e = launch_export(a, (int)(s->t & 1), s->storage, s->layout, s->ns, which, out, st);
  if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(dst, tmp, sizeof(float) * count, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (tmp) s->mem.free(tmp, sizeof(float) * count);
  if (e != cudaSuccess) return cuda_fail(e, "export");
  return LBM_OK;
}

int lbm_get_field(lbm_sim *s, int which, void *dst, int dst_on_device) {
  NvtxRange nvtx_range("lbm_get_field");
  if (!s || !dst) return arg_fail("null argument");
  if (which < LBM_FIELD_RHO_C || which > LBM_FIELD_DRHO_C) return arg_fail("unknown field");
  if (which == LBM_FIELD_RHO_P && s->ns < 3) return arg_fail("no product species in this simulation");
  return export_common(s, which, (float *)dst, dst_on_device, (size_t)s->g->n);
}

int lbm_get_populations(lbm_sim *s, float *dst, int dst_on_device) {
  if (!s || !dst) return arg_fail("null argument");
  return export_common(s, -1, dst, dst_on_device, (size_t)s->ns * kQ * s->g->n);
}

// ---- bounded-wait self-test ---------------------------------------------
// Every CTA counts its arrival, then waits (bounded) until `expected` CTAs
// have arrived: the wait of the batched launch, in isolation.
__global__ void wait_selftest_kernel(BatchSync *sync, unsigned expected, unsigned long long timeout_ns,
                                     int *passed) {
  if (threadIdx.x != 0) return;
  atomicAdd(&sync->done[0], 1u);
  if (wait_counter(&sync->done[0], expected, &sync->timed_out, timeout_ns)) atomicAdd(passed, 1);
}

int lbm_selftest_barrier(int ctas, int expected, double timeout_s, void *stream, int *passed) {
  if (ctas < 1 || ctas > 8 || expected < 1 || expected > 64 || !(timeout_s > 0.0 && timeout_s <= 10.0) || !passed)
    return arg_fail("selftest: 1 <= ctas <= 8, 1 <= expected <= 64, 0 < timeout_s <= 10");
  cudaStream_t st = (cudaStream_t)stream;
  struct Scratch {
    BatchSync sync;
    int passed;
  };
  Scratch *d = nullptr;
  int h_passed = 0, h_flag = 0;
  cudaError_t e = cudaMallocAsync((void **)&d, sizeof(Scratch), st);
  if (e != cudaSuccess) return cuda_fail(e, "selftest alloc");
  e = cudaMemsetAsync(d, 0, sizeof(Scratch), st);
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<ctas, 32, 0, st>>>(&d->sync, (unsigned)expected, (unsigned long long)(timeout_s * 1e9),
                                              &d->passed);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_passed, &d->passed, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_flag, &d->sync.timed_out, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(d, st);
  if (e != cudaSuccess) return cuda_fail(e, "selftest");
  *passed = h_passed;
  if (h_flag) {
    set_error("selftest wait ran past its limit");
    return LBM_ERR_TIMEOUT;
  }
  return LBM_OK;
}

// ---- checkpoint / restore ----------------------------------------------
namespace {
struct StateHeader {
  uint64_t magic;  // "LBMSTATE"
  uint64_t mask_hash;
  uint32_t version;
  int32_t storage, layout, ns, det;
  int32_t modes;  // bit 0: random sputtering matrix; bit 1: barycentric velocity; bit 2: velocity inlet;
                  // bit 3: channel kernel variant; bit 4: species bounce-back
  int64_t n_lat, n_pad, n_nodes, n_nodes_pad, n_blocks, n_flux_slots, plane, nz, t;
  double M0[3];
};
constexpr uint64_t kStateMagic = 0x4554415453424D4CULL;  // "LBMSTATE" little-endian
// 2: carrier and species in separate warp-blocked arrays, reactant and
// product of a slot adjacent
constexpr uint32_t kStateVersion = 2;
static_assert(sizeof(StateHeader) == LBM_STATE_HEADER_BYTES, "state header layout");
struct StatePart {
  void *dev;
  size_t bytes;
};
static std::vector<StatePart> state_parts(const lbm_sim *s) {
  return {{s->f, (size_t)s->ns * kQ * s->n_pad * storage_bytes(s->storage)},
          {s->A, sizeof(acc_t) * 3 * 2 * s->acc_row},
          {s->ub, sizeof(float) * 2 * 2 * 5 * s->g->plane},
          {s->node_cum, sizeof(double) * 2 * s->n_blocks},
          {s->flux_cum, sizeof(double) * 6 * std::max<int64_t>(s->n_flux_slots, 1)}};
}
static StateHeader state_header(const lbm_sim *s) {
  StateHeader h{};
  h.magic = kStateMagic;
  h.mask_hash = s->g->mask_hash;
  h.version = kStateVersion;
  h.storage = s->storage;
  h.layout = s->layout;
  h.ns = s->ns;
  h.det = s->det;
  h.modes = s->rs | (s->bary << 1) | (s->vel_in << 2) | ((s->phys == kPhysChannel) << 3) | (s->sp_bb << 4);
  h.n_lat = s->n_lat;
  h.n_pad = s->n_pad;
  h.n_nodes = s->g->n_nodes;
  h.n_nodes_pad = s->n_nodes_pad;
  h.n_blocks = s->n_blocks;
  h.n_flux_slots = s->n_flux_slots;
  h.plane = s->g->plane;
  h.nz = s->g->nz;
  h.t = s->t;
  for (int k = 0; k < 3; ++k) h.M0[k] = s->M0[k];
  return h;
}
}  // namespace

int lbm_state_size(const lbm_sim *s, size_t *bytes) {
  if (!s || !bytes) return arg_fail("null argument");
  size_t b = sizeof(StateHeader);
  for (auto &p : state_parts(s)) b += p.bytes;
  *bytes = b;
  return LBM_OK;
}

int lbm_get_state(lbm_sim *s, void *dst, size_t n) {
  NvtxRange nvtx_range("lbm_get_state");
  size_t need = 0;
  int rc = lbm_state_size(s, &need);
  if (rc) return rc;
  if (!dst || n < need) return arg_fail("state buffer too small");
  const StateHeader h = state_header(s);
  std::memcpy(dst, &h, sizeof(h));
  char *p = static_cast<char *>(dst) + sizeof(h);
  cudaStream_t st = s->mem.stream;
  for (auto &part : state_parts(s)) {
    LBM_CUDA_TRY(cudaMemcpyAsync(p, part.dev, part.bytes, cudaMemcpyDeviceToHost, st), "get state");
    p += part.bytes;
  }
  LBM_CUDA_TRY(cudaStreamSynchronize(st), "get state sync");
  return LBM_OK;
}

int lbm_set_state(lbm_sim *s, const void *src, size_t n) {
  NvtxRange nvtx_range("lbm_set_state");
  size_t need = 0;
  int rc = lbm_state_size(s, &need);
  if (rc) return rc;
  if (!src || n < need) return arg_fail("state buffer too small");
  StateHeader h;
  std::memcpy(&h, src, sizeof(h));
  StateHeader mine = state_header(s);
  mine.t = h.t;
  for (int k = 0; k < 3; ++k) mine.M0[k] = h.M0[k];
  if (h.magic != kStateMagic || h.version != kStateVersion || std::memcmp(&h, &mine, sizeof(h)) != 0)
    return arg_fail("state does not match this simulation (geometry, storage, layout, species or mode)");
  const char *p = static_cast<const char *>(src) + sizeof(h);
  cudaStream_t st = s->mem.stream;
  for (auto &part : state_parts(s)) {
    LBM_CUDA_TRY(cudaMemcpyAsync(part.dev, p, part.bytes, cudaMemcpyHostToDevice, st), "set state");
    p += part.bytes;
  }
  LBM_CUDA_TRY(cudaStreamSynchronize(st), "set state sync");
  s->t = h.t;
  for (int k = 0; k < 3; ++k) s->M0[k] = h.M0[k];
  return LBM_OK;
}

int lbm_check_status(uint64_t *word) {
  if (!word) return arg_fail("null argument");
#ifdef LBM_CHECKED
  unsigned long long *w = check_word();
  if (!w) return cuda_fail(cudaErrorMemoryAllocation, "check word");
  unsigned long long v = 0;
  LBM_CUDA_TRY(cudaDeviceSynchronize(), "check sync");
  LBM_CUDA_TRY(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost), "check read");
  LBM_CUDA_TRY(cudaMemset(w, 0, sizeof(v)), "check clear");
  *word = v;
  return LBM_OK;
#else
  *word = 0;
  set_error("not a checked build (-DLBM_CHECKED)");
  return LBM_ERR_STATE;
#endif
}

int lbm_warp_counts(const lbm_sim *s, int64_t *counts) {
  if (!s || !counts) return arg_fail("null argument");
  counts[0] = s->n_fast - s->n_uni;
  counts[1] = s->n_uni;
  counts[2] = s->n_wall;
  counts[3] = s->n_gen;
  return LBM_OK;
}

int lbm_sim_info(const lbm_sim *s, int64_t *step, int *storage, int *layout, double *p) {
  if (!s) return arg_fail("null simulation");
  if (step) *step = s->t;
  if (storage) *storage = s->storage;
  if (layout) *layout = s->layout;
  if (p) *p = s->p;
  return LBM_OK;
}

void lbm_destroy(lbm_sim *s) {
  if (!s) return;
  sim_free_all(s);
  cudaStreamSynchronize(s->mem.stream);
  delete s;
}

}  // extern "C"
