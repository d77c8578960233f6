// lbm_observables_noalloc: the observables reduction with its scratch in a
// fixed device array, for callers that cannot allocate device memory.
//
// Who needs it: a caller that hands the library an exact memory budget, such
// as the serving loop that admits simulations by their HBM footprint, or an
// application whose allocator is not safe to call from the thread that polls
// conversion. lbm_observables stages the site map in a temporary device
// buffer; this variant never allocates, so the footprint a caller reserved
// (lbm_footprint) stays the whole story.
//
// The scratch below is a file-scope __device__ array: every GPU that loads
// this library holds it (about 360 KB) until the process exits. All calls on
// all simulations of a device share it, and it keeps the last call's
// contents. Every value a call reads is first written by that same call, so
// nothing needs clearing between calls, but calls that overlap on the GPU
// (two streams, or two host threads at once) race on it and must be
// serialised by the caller.
#include <cmath>
#include <mutex>

#include "lbm_internal.h"

namespace lbm {

constexpr int kNoAllocProfiles = 5;  // rhoC, rhoR, rhoP, phiP, react per plane
constexpr int kNoAllocScalars = 16;
constexpr size_t kNoAllocRows = (size_t)LBM_NOALLOC_MAX_PLANES * kPlaneCols;
constexpr size_t kNoAllocProf = (size_t)kNoAllocProfiles * LBM_NOALLOC_MAX_PLANES;
constexpr size_t kNoAllocDoubles = kNoAllocRows + kNoAllocProf + 8 + kNoAllocScalars;

// [rows: LBM_NOALLOC_MAX_PLANES x kPlaneCols][profiles: 5 x max planes][column totals: 8][scalars: 16]
static __device__ __align__(256) double g_obs_scratch[kNoAllocDoubles];

// Host code cannot use g_obs_scratch's name as a device address: it is a
// host-side stand-in. The device address is looked up once per device and
// kept for the process's life, so the entry point must not be used after a
// reset of the device (cudaDeviceReset), which re-creates the context.
constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static double *g_scratch_dev[kMaxDevices] = {};

static cudaError_t scratch_address(int dev, double **out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_obs_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = (double *)p;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

// One thread: the same sums, in the same order, as lbm_observables does on
// the host, so the two entry points agree to the last bit.
__global__ void noalloc_finish_kernel(double *scr, int nz, int periodic, double react_coef) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double *rows = scr;
  double *prof = scr + kNoAllocRows;
  const double *red = prof + kNoAllocProf;
  double *out = (double *)red + 8;
  double M0 = 0, M1 = 0, M2 = 0, hR = red[0], hP = red[1];
  double bad = 0.0;
  for (int z = 0; z < nz; ++z) {
    const double *row = rows + (size_t)kPlaneCols * z;
    for (int k = 0; k < kPlaneCols; ++k)
      if (row[k] != row[k]) bad = 1.0;
    const bool bc = !periodic && (z == 0 || z == nz - 1);
    if (bc) {
      for (int k = 0; k < kNoAllocProfiles; ++k) prof[(size_t)k * LBM_NOALLOC_MAX_PLANES + z] = 0.0;
      continue;
    }
    M0 += row[0];
    M1 += row[1];
    M2 += row[2];
    hR += row[4];
    hP += row[5];
    for (int k = 0; k < 4; ++k) prof[(size_t)k * LBM_NOALLOC_MAX_PLANES + z] = row[k];
    prof[(size_t)4 * LBM_NOALLOC_MAX_PLANES + z] = react_coef * row[4];
  }
  out[0] = M0;
  out[1] = M1;
  out[2] = M2;
  out[3] = hR;
  out[4] = hP;
  out[5] = rows[(size_t)kPlaneCols * 1 + 1];         // sum rho_R, plane 1
  out[6] = rows[(size_t)kPlaneCols * (nz - 2) + 2];  // sum rho_P, plane nz-2
  out[7] = bad;
  for (int k = 0; k < 6; ++k) out[8 + k] = red[2 + k];  // face flows
}

}  // namespace lbm

using namespace lbm;

extern "C" int lbm_observables_noalloc(lbm_sim *s, lbm_obs *o) {
  if (!s || !o) return LBM_ERR_ARG;
  const lbm_geometry *g = s->g;
  if (g->nz > LBM_NOALLOC_MAX_PLANES) return LBM_ERR_ARG;  // scratch holds LBM_NOALLOC_MAX_PLANES planes
  if (o->site_map) return LBM_ERR_ARG;                      // the site map needs staging: use lbm_observables
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return LBM_ERR_CUDA;
  const int dev = g->device;
  if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_ARG;
  if (dev != prev && cudaSetDevice(dev) != cudaSuccess) return LBM_ERR_CUDA;
  double *scr = nullptr;
  cudaError_t e = scratch_address(dev, &scr);
  const cudaStream_t st = s->mem.stream;
  double buf[kNoAllocScalars] = {0};
  if (e == cudaSuccess) {
    ObsArgs oa{};
    oa.s = make_args(s);
    oa.parity = (int)(s->t & 1);
    oa.lat_plane = s->layout == LBM_LAYOUT_DENSE ? g->cell_plane_d : g->fl_plane_d;
    oa.node_plane = g->node_plane_d;
    oa.plane_sums = scr;
    e = launch_plane_sums(oa, s->storage, s->layout, s->ns, st);
  }
  double *red = scr + kNoAllocRows + kNoAllocProf;
  if (e == cudaSuccess) e = launch_sum_columns(s->node_cum, s->n_blocks, 2, red, st);
  if (e == cudaSuccess) {
    if (g->bc != LBM_BC_PERIODIC && s->n_flux_slots > 0)
      e = launch_sum_columns(s->flux_cum, s->n_flux_slots, 6, red + 2, st);
    else
      e = cudaMemsetAsync(red + 2, 0, sizeof(double) * 6, st);
  }
  const double coef = s->p * s->prm.pS_R;
  if (e == cudaSuccess) {
    noalloc_finish_kernel<<<1, 1, 0, st>>>(scr, g->nz, g->bc == LBM_BC_PERIODIC, coef);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf, red + 8, sizeof(double) * 14, cudaMemcpyDeviceToHost, st);
  double *dst[kNoAllocProfiles] = {o->rhoC_z, o->rhoR_z, o->rhoP_z, o->phiP_z, o->react_z};
  for (int k = 0; k < kNoAllocProfiles && e == cudaSuccess; ++k)
    if (dst[k])
      e = cudaMemcpyAsync(dst[k], scr + kNoAllocRows + (size_t)k * LBM_NOALLOC_MAX_PLANES, sizeof(double) * g->nz,
                          cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (dev != prev) cudaSetDevice(prev);
  if (e != cudaSuccess) return LBM_ERR_CUDA;

  const double p = s->p, pSR = s->prm.pS_R, pSP = s->prm.pS_P;
  const double M[3] = {buf[0], buf[1], buf[2]};
  const double hitsR = buf[3], hitsP = buf[4], mRin = buf[5], mPout = buf[6];
  o->step = s->t;
  o->M_C = M[0];
  o->M_R = M[1];
  o->M_P = M[2];
  o->eta = mRin != 0.0 ? mPout / mRin : 0.0;
  o->in_C = buf[8];
  o->in_R = buf[9];
  o->in_P = buf[10];
  o->out_C = buf[11];
  o->out_R = buf[12];
  o->out_P = buf[13];
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
  if (buf[7] != 0.0 || !(M[0] > 0.0)) return LBM_ERR_DIVERGED;
  return LBM_OK;
}
