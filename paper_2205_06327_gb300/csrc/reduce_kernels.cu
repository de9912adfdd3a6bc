// Deterministic reductions: the object gradient as an owner-computes tiled
// accumulation (the one-GPU form of the image-gradient decomposition of
// Sec. III), the probe gradient, the FP64 loss, and the small vector kernels
// of the gradient-descent step.
//
// Object gradient (Eq. 2 with the locality of Sec. III): slice s of dF/dO is
// sum_i conj(psi_{i,s}) * g_phi_{i,s} placed at window i.  The object is
// tessellated into tiles; one block owns one (tile, slice), walks the
// positions whose window meets its tile in ascending order and sums their
// contributions in registers.  Every output pixel therefore has exactly one
// writer and a fixed summation order: no atomics, bit-reproducible.
#include "internal.h"
#include "../../include/ptycho.h"

namespace ptycho {

namespace {

__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }

constexpr int kAccThreads = 256;

// Accumulation shape: positions whose loads are in flight together, and
// resident blocks per SM the kernel is compiled for.
#ifndef PTYCHO_ACC_UNROLL
#define PTYCHO_ACC_UNROLL 4
#endif
#ifndef PTYCHO_ACC_MIN_BLOCKS
#define PTYCHO_ACC_MIN_BLOCKS 2
#endif
constexpr int kAccUnroll = PTYCHO_ACC_UNROLL;
constexpr int kAccPPT = 4;     // pixels per thread per pixel group

// One block owns one (tile, slice).  The tile's pixels are processed in
// groups of kAccPPT * 256; for each group the block walks the positions whose
// window meets the group's rows, in ascending order.
__global__ void __launch_bounds__(kAccThreads, PTYCHO_ACC_MIN_BLOCKS) k_accum_obj_grad(const AccumArgs a) {
  __shared__ int2 lpos[kAccThreads];
  __shared__ int lidx[kAccThreads];
  __shared__ int wcount[kAccThreads / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int z = blockIdx.z;  // slice s_begin + z
  const int s = a.s_begin + z;
  const int M = a.M;
  const int ty0 = blockIdx.y * a.tile_h, tx0 = blockIdx.x * a.tile_w;
  const int th = min(a.tile_h, a.H - ty0), tw = min(a.tile_w, a.W - tx0);
  const int npix = th * tw;
  const size_t MM = (size_t)M * M;
  const float2* gphi_s = a.ws_gphi + (size_t)(a.seg_slots ? z : s) * a.ws_n * MM;
  const float2* psi_s =
      s > 0 && !a.patch_mode ? a.ws_psi + (size_t)(a.seg_slots ? z : s - 1) * a.ws_n * MM : nullptr;
  float2* out = a.grad_obj + (size_t)s * a.H * a.W;
  constexpr int GROUP = kAccPPT * kAccThreads;

  for (int pg0 = 0; pg0 < npix; pg0 += GROUP) {
    // Pixel k of this thread: p = pg0 + t + 256 k in the tile, row-major.
    int rowk[kAccPPT], colk[kAccPPT];
    float2 acc[kAccPPT];
#pragma unroll
    for (int k = 0; k < kAccPPT; ++k) {
      const int p = pg0 + t + kAccThreads * k;
      rowk[k] = p < npix ? p / tw : (1 << 28);
      colk[k] = p < npix ? p % tw : 0;
      acc[k] = make_float2(0.f, 0.f);
    }
    const int gy0 = ty0 + pg0 / tw;
    const int gy1 = ty0 + min(npix - 1, pg0 + GROUP - 1) / tw + 1;  // rows [gy0, gy1)

    for (int base = 0; base < a.n_pos; base += kAccThreads) {
      // Positions of this batch whose window meets the group, compacted in
      // ascending order (ballot + warp prefix): the summation order.
      const int il = base + t;
      bool hit = false;
      int2 r = make_int2(0, 0);
      if (il < a.n_pos) {
        r = a.pos[a.pos_begin + il];
        const bool ok = r.x >= 0 && r.y >= 0 && r.x <= a.H - M && r.y <= a.W - M;
        hit = ok && r.x < gy1 && r.x + M > gy0 && r.y < tx0 + tw && r.y + M > tx0;
      }
      const unsigned b = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) wcount[w] = __popc(b);
      __syncthreads();
      int off = 0, total = 0;
#pragma unroll
      for (int k = 0; k < kAccThreads / 32; ++k) {
        off += k < w ? wcount[k] : 0;
        total += wcount[k];
      }
      if (hit) {
        const int slot = off + __popc(b & ((1u << lane) - 1u));
        lpos[slot] = r;
        lidx[slot] = il;
      }
      __syncthreads();
      for (int j0 = 0; j0 < total; j0 += kAccUnroll) {
        // Issue the loads of up to kAccUnroll positions, then add them in
        // order.  Pixels outside a window load zeros, whose product adds
        // exactly nothing.
        float2 pv[kAccUnroll][kAccPPT], gv[kAccUnroll][kAccPPT];
#pragma unroll
        for (int u = 0; u < kAccUnroll; ++u) {
          const int j = j0 + u;
          const bool live = j < total;
          const int2 rr = lpos[live ? j : 0];
          const int i = lidx[live ? j : 0];
          const int oy0 = ty0 - rr.x, ox0 = tx0 - rr.y;
          const float2* gp = gphi_s + (size_t)i * MM;
          const float2* pp = s > 0 && !a.patch_mode ? psi_s + (size_t)i * MM : a.probe;
          if (a.patch_mode) {  // finished patches conj(psi) g_phi
#pragma unroll
            for (int k = 0; k < kAccPPT; ++k) {
              const int oy = oy0 + rowk[k], ox = ox0 + colk[k];
              const bool in = live && (unsigned)oy < (unsigned)M && (unsigned)ox < (unsigned)M;
              pv[u][k] = in ? ld_stream(gp + oy * M + ox) : make_float2(0.f, 0.f);
            }
          } else {
#pragma unroll
            for (int k = 0; k < kAccPPT; ++k) {
              const int oy = oy0 + rowk[k], ox = ox0 + colk[k];
              const bool in = live && (unsigned)oy < (unsigned)M && (unsigned)ox < (unsigned)M;
              const int idx = in ? oy * M + ox : 0;
              pv[u][k] = in ? (s > 0 ? ld_stream(pp + idx) : __ldg(pp + idx)) : make_float2(0.f, 0.f);
              gv[u][k] = in ? ld_stream(gp + idx) : make_float2(0.f, 0.f);
            }
          }
        }
        if (a.patch_mode) {
#pragma unroll
          for (int u = 0; u < kAccUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kAccPPT; ++k) {
              acc[k].x += pv[u][k].x;
              acc[k].y += pv[u][k].y;
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < kAccUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kAccPPT; ++k) {
              const float2 p = pv[u][k], g = gv[u][k];
              acc[k].x = fmaf(p.x, g.x, fmaf(p.y, g.y, acc[k].x));
              acc[k].y = fmaf(p.x, g.y, fmaf(-p.y, g.x, acc[k].y));
            }
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kAccPPT; ++k) {
      if (rowk[k] < th) {
        float2* o = out + (size_t)(ty0 + rowk[k]) * a.W + (tx0 + colk[k]);
        float2 val = acc[k];
        if (a.accumulate) {
          const float2 prev = *o;
          val.x += prev.x;
          val.y += prev.y;
        }
        *o = val;
      }
    }
  }
}

// part[sp][pix] = sum over positions of split sp (ascending) of ws_gp[i][pix]
__global__ void k_probe_grad_part(const float2* __restrict__ ws_gp, int n_pos, int MM, int n_split,
                                  float2* __restrict__ part) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  const int sp = blockIdx.y;
  if (pix >= MM) return;
  const int per = (n_pos + n_split - 1) / n_split;
  const int i0 = sp * per, i1 = min(n_pos, i0 + per);
  float2 acc = make_float2(0.f, 0.f);
  for (int i = i0; i < i1; ++i) {
    const float2 g = __ldcs(ws_gp + (size_t)i * MM + pix);
    acc.x += g.x;
    acc.y += g.y;
  }
  part[(size_t)sp * MM + pix] = acc;
}

__global__ void k_probe_grad_final(const float2* __restrict__ part, int MM, int n_split,
                                   float2* __restrict__ gp, int accumulate) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= MM) return;
  float2 acc = accumulate ? gp[pix] : make_float2(0.f, 0.f);
  for (int sp = 0; sp < n_split; ++sp) {
    const float2 g = part[(size_t)sp * MM + pix];
    acc.x += g.x;
    acc.y += g.y;
  }
  gp[pix] = acc;
}

// Fixed-order FP64 sum of n values into acc[0] (one block).
__global__ void k_loss_accum(const double* __restrict__ part, int n, double* acc, int accumulate) {
  __shared__ double sh[256];
  const int t = threadIdx.x;
  double s = 0.0;
  for (int i = t; i < n; i += 256) s += part[i];
  sh[t] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) sh[t] += sh[t + h];
    __syncthreads();
  }
  if (t == 0) acc[0] = (accumulate ? acc[0] : 0.0) + sh[0];
}

__global__ void k_axpy(float2* y, const float2* __restrict__ x, const float2* base, float alpha, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 b = base[i], d = x[i];
    y[i] = make_float2(fmaf(alpha, d.x, b.x), fmaf(alpha, d.y, b.y));
  }
}

// Sum of |x|^2 in FP64: per-block partials over a fixed index assignment.
__global__ void k_norm2_part(const float2* __restrict__ x, size_t n, double* part) {
  __shared__ double sh[256];
  const int t = threadIdx.x;
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)256 + t; i < n; i += (size_t)gridDim.x * 256) {
    const float2 v = x[i];
    s += (double)v.x * v.x + (double)v.y * v.y;
  }
  sh[t] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) sh[t] += sh[t + h];
    __syncthreads();
  }
  if (t == 0) part[blockIdx.x] = sh[0];
}

// O = exp(i sigma V) for a real potential V (Sec. II-B's unknown).
__global__ void k_potential_to_transmission(const float* __restrict__ V, float2* __restrict__ O, float sigma,
                                            size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float sn, cs;
    sincosf(sigma * V[i], &sn, &cs);
    O[i] = make_float2(cs, sn);
  }
}

// dF/dV = sigma * Im(conj(O) dF/dO) for O = exp(i sigma V), V real.
__global__ void k_potential_grad(const float2* __restrict__ O, const float2* __restrict__ g, float* __restrict__ gV,
                                 float sigma, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 o = O[i], d = g[i];
    gV[i] = sigma * fmaf(o.x, d.y, -o.y * d.x);
  }
}

__global__ void k_check_positions(const int2* __restrict__ pos, int n, int M, int H, int W, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int2 r = pos[i];
  if (r.x < 0 || r.y < 0 || r.x > H - M || r.y > W - M) *status = PTYCHO_ERR_POSITION;
}

}  // namespace

cudaError_t launch_accum_obj_grad(const AccumArgs& a, cudaStream_t st) {
  const int ns = a.n_slices > 0 ? a.n_slices : a.S - a.s_begin;
  if (a.s_begin < 0 || ns <= 0 || a.s_begin + ns > a.S) return cudaErrorInvalidValue;
  const dim3 grid((a.W + a.tile_w - 1) / a.tile_w, (a.H + a.tile_h - 1) / a.tile_h, ns);
  k_accum_obj_grad<<<grid, kAccThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_probe_grad(const float2* ws_gp, int n_pos, int M, float2* part, int n_split,
                              float2* grad_probe, int accumulate, cudaStream_t st) {
  const int MM = M * M;
  const dim3 g1((MM + 255) / 256, n_split);
  k_probe_grad_part<<<g1, 256, 0, st>>>(ws_gp, n_pos, MM, n_split, part);
  k_probe_grad_final<<<(MM + 255) / 256, 256, 0, st>>>(part, MM, n_split, grad_probe, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_loss_accum(const double* loss_part, int n, double* acc, int accumulate, cudaStream_t st) {
  k_loss_accum<<<1, 256, 0, st>>>(loss_part, n, acc, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_axpy(float2* y, const float2* x, const float2* base, double alpha, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + 255) / 256;
  k_axpy<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(y, x, base, (float)alpha, n);
  return cudaGetLastError();
}

cudaError_t launch_norm2(const float2* x, size_t n, double* part, int n_part, double* out, int slot,
                         cudaStream_t st) {
  k_norm2_part<<<n_part, 256, 0, st>>>(x, n, part);
  k_loss_accum<<<1, 256, 0, st>>>(part, n_part, out + slot, 0);
  return cudaGetLastError();
}

cudaError_t launch_potential_to_transmission(const float* V, float2* O, double sigma, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + 255) / 256;
  k_potential_to_transmission<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(V, O, (float)sigma, n);
  return cudaGetLastError();
}

cudaError_t launch_potential_grad(const float2* O, const float2* g, float* gV, double sigma, size_t n,
                                  cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + 255) / 256;
  k_potential_grad<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(O, g, gV, (float)sigma, n);
  return cudaGetLastError();
}

cudaError_t launch_check_positions(const int2* pos, int n, int M, int H, int W, int* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_check_positions<<<(n + 255) / 256, 256, 0, st>>>(pos, n, M, H, W, status);
  return cudaGetLastError();
}

}  // namespace ptycho
