// Geometry: the synthetic np-Au stand-in (host, OpenMP) and the derived
// integer structures on the device.
//
// The paper's own samples are grown from random 30 nm disks to a porosity of
// 0.70 (Sec. 2.1). Here the porous slab is a thresholded integer Gaussian
// random field with the requested porosity and correlation length; every
// solid cell touching gas is a catalytic node with b(x) active links
// (Appendix, after Eq. f_P_in). A caller mask may also mark inert solid
// (value 2): it bounces every array back and is never a node.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------------------
// Host: integer Gaussian random field and threshold
// ---------------------------------------------------------------------------
static inline uint64_t splitmix64(uint64_t x) {
  // SplitMix64 (Steele, Lea, Flood 2014): first output for state x
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static int odd_box_width(double corr_len) {
  // nearest odd integer to sqrt(2 l^2 + 1): three box passes of width W have
  // variance 3 (W^2 - 1) / 12 ~ l^2 / 2, the Gaussian kernel of covariance
  // exp(-r^2 / (2 l^2))
  const double t = std::sqrt(2.0 * corr_len * corr_len + 1.0);
  int w = 1;
  double best = std::fabs(t - 1.0);
  for (int k = 3; k <= (int)t + 3; k += 2) {
    const double d = std::fabs(t - k);
    if (d < best) {  // strict: ties keep the smaller width
      best = d;
      w = k;
    }
  }
  return w;
}

// Periodic running-window sum of odd width W along one axis, exact in int64.
// Along x each row slides on its own; along y and z whole contiguous x-rows
// slide together, so every access walks memory in order.
static void box_axis(std::vector<int64_t> &v, std::vector<int64_t> &tmp, int nx, int ny, int nz, int axis, int W) {
  const int r = W / 2;
  const int64_t plane = (int64_t)nx * ny;
  if (axis == 0) {
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < (int64_t)ny * nz; ++row) {
      const int64_t base = row * nx;
      auto at = [&](int k) { return v[base + ((k % nx) + nx) % nx]; };
      int64_t s = 0;
      for (int d = -r; d <= r; ++d) s += at(d);
      for (int k = 0; k < nx; ++k) {
        tmp[base + k] = s;
        s += at(k + r + 1) - at(k - r);
      }
    }
  } else {
    const int m = axis == 1 ? ny : nz;
    const int64_t stride = axis == 1 ? nx : plane;       // distance between successive lines
    const int64_t outer = axis == 1 ? nz : ny;            // independent groups
    const int64_t outer_stride = axis == 1 ? plane : nx;
#pragma omp parallel
    {
      std::vector<int64_t> acc(nx);
#pragma omp for schedule(static)
      for (int64_t o = 0; o < outer; ++o) {
        const int64_t base = o * outer_stride;
        auto row = [&](int k) { return &v[base + (int64_t)(((k % m) + m) % m) * stride]; };
        std::fill(acc.begin(), acc.end(), 0);
        for (int d = -r; d <= r; ++d) {
          const int64_t *p = row(d);
          for (int x = 0; x < nx; ++x) acc[x] += p[x];
        }
        for (int k = 0; k < m; ++k) {
          int64_t *out = &tmp[base + (int64_t)k * stride];
          for (int x = 0; x < nx; ++x) out[x] = acc[x];
          const int64_t *add = row(k + r + 1), *sub = row(k - r);
          for (int x = 0; x < nx; ++x) acc[x] += add[x] - sub[x];
        }
      }
    }
  }
  v.swap(tmp);
}

void grf_mask(int nx, int ny, int nz, int z0, int z1, double porosity, double corr_len, uint64_t seed,
              uint8_t *mask) {
  const int64_t n = (int64_t)nx * ny * nz, plane = (int64_t)nx * ny;
  std::vector<int64_t> v(n), tmp(n);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; ++c) {
    int64_t s = 0;
    for (uint64_t k = 0; k < 12; ++k) s += (int64_t)(splitmix64(seed ^ ((uint64_t)c * 12 + k)) >> 48);
    v[c] = s - 12 * 32768;
  }
  const int W = odd_box_width(corr_len);
  for (int axis = 0; axis < 3; ++axis)
    for (int pass = 0; pass < 3; ++pass) box_axis(v, tmp, nx, ny, nz, axis, W);
  std::vector<int64_t>().swap(tmp);

  std::memset(mask, 0, (size_t)n);
  const int64_t n_slab = plane * (z1 - z0);
  if (n_slab <= 0) return;
  const int64_t K = (int64_t)std::llrint(porosity * (double)n_slab);  // ties to even
  struct KV {
    int64_t v, i;
  };
  std::vector<KV> kv(n_slab);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n_slab; ++k) {
    const int64_t c = (int64_t)z0 * plane + k;
    kv[k] = {v[c], c};
  }
  auto less = [](const KV &a, const KV &b) { return a.v < b.v || (a.v == b.v && a.i < b.i); };
  if (K > 0 && K < n_slab) std::nth_element(kv.begin(), kv.begin() + K, kv.end(), less);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n_slab; ++k) mask[kv[k].i] = (k < K) ? 0 : 1;
}

double chord_length(int nx, int ny, int nz, int z0, int z1, const uint8_t *mask) {
  const int64_t plane = (int64_t)nx * ny;
  int64_t nf = 0, runs = 0;
#pragma omp parallel for reduction(+ : nf, runs) schedule(static)
  for (int z = z0; z < z1; ++z) {
    for (int y = 0; y < ny; ++y) {
      bool row_all = true;
      for (int x = 0; x < nx; ++x) {
        const int64_t c = z * plane + (int64_t)y * nx + x;
        if (mask[c]) {
          row_all = false;
          continue;
        }
        ++nf;
        runs += mask[c - x + (x == 0 ? nx - 1 : x - 1)];
        runs += mask[z * plane + (int64_t)(y == 0 ? ny - 1 : y - 1) * nx + x];
        runs += (z == z0) ? 1 : mask[c - plane];
      }
      runs += row_all;
    }
    for (int x = 0; x < nx; ++x) {
      bool col_all = true;
      for (int y = 0; y < ny && col_all; ++y) col_all = !mask[z * plane + (int64_t)y * nx + x];
      runs += col_all;
    }
  }
  if (nf == 0 || runs == 0) return 0.0;
  return 3.0 * (double)nf / (double)runs;
}

// ---------------------------------------------------------------------------
// Device: b(x), numbering, neighbour masks
// ---------------------------------------------------------------------------
struct GeoArgs {
  const uint8_t *mask;
  int32_t nx, ny, nz, per_z;
};

__device__ __forceinline__ int64_t geo_nbr(const GeoArgs &g, int x, int y, int z, int dx, int dy, int dz) {
  int xx = x + dx, yy = y + dy, zz = z + dz;
  xx = xx < 0 ? xx + g.nx : (xx >= g.nx ? xx - g.nx : xx);
  yy = yy < 0 ? yy + g.ny : (yy >= g.ny ? yy - g.ny : yy);
  if (zz < 0 || zz >= g.nz) {
    if (!g.per_z) return -1;
    zz = zz < 0 ? zz + g.nz : zz - g.nz;
  }
  return ((int64_t)zz * g.ny + yy) * g.nx + xx;
}

// b(c) for catalytic solid cells (fluid cells at c - c_j; 0 for inert solid),
// and the 18-bit masks: for fluid cells, bit i set when c + c_i is solid (the
// targets that bounce back or sputter); for solid cells, bit i set when
// c + c_i is fluid (the node's active outgoing links, from which the random
// sputtering matrix draws). Also counts fluid->catalytic links.
__global__ void classify_kernel(GeoArgs g, int32_t *b, uint32_t *nbm_dense, unsigned long long *n_links) {
  const int64_t n = (int64_t)g.nx * g.ny * g.nz;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int links = 0;
  if (c < n) {
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int z = (int)(c / plane);
    const int y = (int)((c - z * plane) / g.nx);
    const int x = (int)(c - z * plane - (int64_t)y * g.nx);
    if (g.mask[c]) {
      int cnt = 0;
      uint32_t out = 0;
#pragma unroll
      for (int j = 1; j < kQ; ++j) {
        const int64_t s = geo_nbr(g, x, y, z, -cx(j), -cy(j), -cz(j));
        cnt += (s >= 0 && !g.mask[s]) ? 1 : 0;
        const int64_t t = geo_nbr(g, x, y, z, cx(j), cy(j), cz(j));
        if (t >= 0 && !g.mask[t]) out |= 1u << j;
      }
      b[c] = g.mask[c] == 1 ? cnt : 0;
      nbm_dense[c] = out;
    } else {
      uint32_t m = 0;
#pragma unroll
      for (int i = 1; i < kQ; ++i) {
        const int64_t t = geo_nbr(g, x, y, z, cx(i), cy(i), cz(i));
        if (t >= 0 && g.mask[t]) {
          m |= 1u << i;
          links += g.mask[t] == 1;
        }
      }
      b[c] = 0;
      nbm_dense[c] = m;
    }
  }
  // integer sum: order-independent
  for (int o = 16; o > 0; o >>= 1) links += __shfl_down_sync(0xffffffffu, links, o);
  if ((threadIdx.x & 31) == 0 && links) atomicAdd(n_links, (unsigned long long)links);
}

// per-plane counts of fluid cells and catalytic nodes: one block per plane
__global__ void plane_count_kernel(GeoArgs g, const int32_t *b, int64_t *fl_cnt, int64_t *node_cnt) {
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t base = (int64_t)blockIdx.x * plane;
  long long f = 0, s = 0;
  for (int64_t k = threadIdx.x; k < plane; k += blockDim.x) {
    const int64_t c = base + k;
    if (g.mask[c])
      s += b[c] > 0;
    else
      f += 1;
  }
  __shared__ long long shf[32], shs[32];
  for (int o = 16; o > 0; o >>= 1) {
    f += __shfl_down_sync(0xffffffffu, f, o);
    s += __shfl_down_sync(0xffffffffu, s, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    shf[wid] = f;
    shs[wid] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tf = 0, ts = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tf += shf[w];
      ts += shs[w];
    }
    fl_cnt[blockIdx.x] = tf;
    node_cnt[blockIdx.x] = ts;
  }
}

// Numbering, one block per plane, tiles of blockDim cells, ranks from a
// ballot/popc block scan:
//   - catalytic nodes in linear order;
//   - lattice entries of the fluid cells (fluid-only addressing): within each
//     plane first the cells with no solid neighbour, then the cells touching
//     a solid, each group in linear order. The second group then fills warps
//     of its own, and the warps of the first take the fast path, instead of
//     one wall cell sending its whole warp of 32 down the general one. (The
//     exported fluid index is the linear-order numbering, formed from the
//     mask on export.)
// pass 0 numbers the nodes and the first group, pass 1 the second group.
__global__ void number_kernel(GeoArgs g, const int32_t *b, const int64_t *fl_plane, const int64_t *node_plane,
                              int32_t *idx, int32_t *fcell, float *inv_b, int32_t *node_cell,
                              const uint32_t *nbm_dense, uint32_t *nbm_fluid) {
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t base = (int64_t)blockIdx.x * plane;
  int64_t fl_off = fl_plane[blockIdx.x], nd_off = node_plane[blockIdx.x];
  __shared__ int wf[32], ws[32];
  __shared__ int64_t tot_f, tot_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int pass = 0; pass < 2; ++pass) {
    for (int64_t t0 = 0; t0 < plane; t0 += blockDim.x) {
      const int64_t k = t0 + threadIdx.x;
      const bool in = k < plane;
      const int64_t c = base + k;
      const bool fl = in && !g.mask[c];
      const bool isf = fl && ((nbm_dense[c] != 0) == (pass == 1));
      const bool iss = pass == 0 && in && g.mask[c] && b[c] > 0;
      const unsigned bf = __ballot_sync(0xffffffffu, isf), bs = __ballot_sync(0xffffffffu, iss);
      const unsigned lt = (1u << lane) - 1u;
      if (lane == 0) {
        wf[wid] = __popc(bf);
        ws[wid] = __popc(bs);
      }
      __syncthreads();
      int pf = 0, ps = 0;
      for (int w = 0; w < wid; ++w) {
        pf += wf[w];
        ps += ws[w];
      }
      if (isf) {
        const int64_t r = fl_off + pf + __popc(bf & lt);
        idx[c] = (int32_t)r;
        fcell[r] = (int32_t)c;
        nbm_fluid[r] = nbm_dense[c];
      } else if (iss) {
        const int64_t r = nd_off + ps + __popc(bs & lt);
        idx[c] = (int32_t)r;
        inv_b[r] = 1.0f / (float)b[c];
        node_cell[r] = (int32_t)c;
      } else if (pass == 0 && in && g.mask[c]) {
        idx[c] = -1;
      }
      if (threadIdx.x == 0) {
        int sf = 0, ss = 0;
        for (int w = 0; w < nw; ++w) {
          sf += wf[w];
          ss += ws[w];
        }
        tot_f = sf;
        tot_s = ss;
      }
      __syncthreads();
      fl_off += tot_f;
      nd_off += tot_s;
      __syncthreads();
    }
  }
}

cudaError_t build_structures(lbm_geometry *g, cudaStream_t st) {
  GeoArgs ga{g->mask, g->nx, g->ny, g->nz, g->bc == LBM_BC_PERIODIC};
  const int64_t n = g->n;
  unsigned long long *d_links = (unsigned long long *)g->mem.alloc(sizeof(unsigned long long));
  int64_t *d_cnt = (int64_t *)g->mem.alloc(sizeof(int64_t) * 2 * g->nz);
  // the two counters go back to the allocator on every exit (stream-ordered)
  struct Scratch {
    lbm_geometry *g;
    unsigned long long *links;
    int64_t *cnt;
    ~Scratch() {
      g->mem.free(links, sizeof(unsigned long long));
      g->mem.free(cnt, sizeof(int64_t) * 2 * g->nz);
    }
  } scratch{g, d_links, d_cnt};
  if (!d_links || !d_cnt) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMemsetAsync(d_links, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  classify_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ga, g->b, g->nbm_dense, d_links);
  plane_count_kernel<<<g->nz, 512, 0, st>>>(ga, g->b, d_cnt, d_cnt + g->nz);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  std::vector<int64_t> cnt(2 * g->nz);
  unsigned long long links = 0;
  if ((e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int64_t) * 2 * g->nz, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(&links, d_links, sizeof(links), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  g->fl_plane_h = new int64_t[g->nz + 1];
  g->node_plane_h = new int64_t[g->nz + 1];
  g->fl_plane_h[0] = g->node_plane_h[0] = 0;
  for (int z = 0; z < g->nz; ++z) {
    g->fl_plane_h[z + 1] = g->fl_plane_h[z] + cnt[z];
    g->node_plane_h[z + 1] = g->node_plane_h[z] + cnt[g->nz + z];
  }
  g->n_fluid = g->fl_plane_h[g->nz];
  g->n_nodes = g->node_plane_h[g->nz];
  g->n_links = (int64_t)links;
  g->nbm_fluid = (uint32_t *)g->mem.alloc(sizeof(uint32_t) * std::max<int64_t>(g->n_fluid, 1));
  g->fcell = (int32_t *)g->mem.alloc(sizeof(int32_t) * std::max<int64_t>(g->n_fluid, 1));
  g->inv_b = (float *)g->mem.alloc(sizeof(float) * std::max<int64_t>(g->n_nodes, 1));
  g->node_cell = (int32_t *)g->mem.alloc(sizeof(int32_t) * std::max<int64_t>(g->n_nodes, 1));
  g->fl_plane_d = (int64_t *)g->mem.alloc(sizeof(int64_t) * (g->nz + 1));
  g->node_plane_d = (int64_t *)g->mem.alloc(sizeof(int64_t) * (g->nz + 1));
  g->cell_plane_d = (int64_t *)g->mem.alloc(sizeof(int64_t) * (g->nz + 1));
  if (!g->nbm_fluid || !g->fcell || !g->inv_b || !g->node_cell || !g->fl_plane_d || !g->node_plane_d || !g->cell_plane_d)
    return cudaErrorMemoryAllocation;
  std::vector<int64_t> cp(g->nz + 1);
  for (int z = 0; z <= g->nz; ++z) cp[z] = (int64_t)z * g->plane;
  if ((e = cudaMemcpyAsync(g->fl_plane_d, g->fl_plane_h, sizeof(int64_t) * (g->nz + 1), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(g->node_plane_d, g->node_plane_h, sizeof(int64_t) * (g->nz + 1), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(g->cell_plane_d, cp.data(), sizeof(int64_t) * (g->nz + 1), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  number_kernel<<<g->nz, 1024, 0, st>>>(ga, g->b, g->fl_plane_d, g->node_plane_d, g->idx, g->fcell, g->inv_b,
                                        g->node_cell, g->nbm_dense, g->nbm_fluid);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

}  // namespace lbm
