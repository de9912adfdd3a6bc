// Generic-window slice chain: any probe window M = 2^a 3^b (8 <= M <= 4096)
// that the register-resident kernels do not cover (they take M = 64, 128).
//
// The chunk's positions advance through the multislice model (Sec. II-B)
// together, slice by slice: their waves live in a global buffer wv[n][M][M],
// every 2-D FFT is a batched pass over rows then a batched pass over columns
// (mixed radix 4/2/3 Stockham autosort in shared memory, natural order, exact
// inverse by conjugation), and pointwise kernels apply the transmission, the
// Fresnel factor, the amplitude residual of Eq. 1 and their adjoints.  The
// workspace it fills (entering waves, exit-wave gradients, probe-gradient
// parts, loss parts) has the layout of the register-resident kernels, so the
// tiled reductions are shared.
#include "../../include/ptycho.h"
#include "internal.h"

namespace ptycho {

namespace {

__device__ __forceinline__ float2 gcmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 gcmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// Small DFTs (natural order), forward kernel exp(-2 pi i n k / R), inverse its conjugate.
template <bool INV>
__device__ __forceinline__ void dft_small(float2 (&x)[4], int R) {
  if (R == 2) {
    const float2 a = x[0], b = x[1];
    x[0] = make_float2(a.x + b.x, a.y + b.y);
    x[1] = make_float2(a.x - b.x, a.y - b.y);
  } else if (R == 3) {
    // X1 = t2 -+ i s3 (b - c), X2 = t2 +- i s3 (b - c), t2 = a - (b + c)/2
    const float s3 = 0.86602540378443864676f;
    const float2 a = x[0], b = x[1], c = x[2];
    const float2 t1 = make_float2(b.x + c.x, b.y + c.y);
    const float2 t2 = make_float2(fmaf(-0.5f, t1.x, a.x), fmaf(-0.5f, t1.y, a.y));
    const float2 d = make_float2(s3 * (b.x - c.x), s3 * (b.y - c.y));  // s3 (b - c)
    // -i d = (d.y, -d.x)
    const float2 mid = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
    x[0] = make_float2(a.x + t1.x, a.y + t1.y);
    x[1] = make_float2(t2.x + mid.x, t2.y + mid.y);
    x[2] = make_float2(t2.x - mid.x, t2.y - mid.y);
  } else {  // R == 4
    const float2 t0 = make_float2(x[0].x + x[2].x, x[0].y + x[2].y);
    const float2 t1 = make_float2(x[0].x - x[2].x, x[0].y - x[2].y);
    const float2 t2 = make_float2(x[1].x + x[3].x, x[1].y + x[3].y);
    const float2 u = make_float2(x[1].x - x[3].x, x[1].y - x[3].y);
    const float2 t3 = INV ? make_float2(-u.y, u.x) : make_float2(u.y, -u.x);  // -+ i (x1 - x3)
    x[0] = make_float2(t0.x + t2.x, t0.y + t2.y);
    x[2] = make_float2(t0.x - t2.x, t0.y - t2.y);
    x[1] = make_float2(t1.x + t3.x, t1.y + t3.y);
    x[3] = make_float2(t1.x - t3.x, t1.y - t3.y);
  }
}

// Batched 1-D FFT of length M over L lines per block: rows (element stride 1)
// or columns (element stride M) of the waves.  Stockham autosort: at a stage
// of radix R after spans Ns, butterfly j takes x[j + t N/R], twiddles it by
// w_{Ns R}^{t (j mod Ns)}, and writes y[(j / Ns) Ns R + j mod Ns + t Ns].
template <bool INV>
__global__ void __launch_bounds__(256) k_gm_fft(float2* __restrict__ data, int M, int L, int cols, GmPlan plan,
                                                const float2* __restrict__ tw) {
  extern __shared__ float2 gsm[];
  float2* A = gsm;
  float2* B = gsm + (size_t)L * M;
  float2* T = B + (size_t)L * M;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int k = t; k < M; k += nt) T[k] = tw[k];
  const size_t MM = (size_t)M * M;
  const int g0 = blockIdx.x * L;  // first line of this block (L divides M)
  const size_t wave = (size_t)(g0 / M);
  const int l0 = g0 % M;
  float2* base = data + wave * MM;
  const int n = L * M;
  if (cols) {
    for (int idx = t; idx < n; idx += nt) {
      const int p = idx / L, li = idx % L;
      A[li * M + p] = base[(size_t)p * M + l0 + li];
    }
  } else {
    for (int idx = t; idx < n; idx += nt) A[idx] = base[(size_t)l0 * M + idx];
  }
  __syncthreads();
  float2* src = A;
  float2* dst = B;
  int Ns = 1;
  for (int st = 0; st < plan.n; ++st) {
    const int R = plan.r[st];
    const int nb = M / R;
    const int tstep = M / (Ns * R);
    for (int idx = t; idx < L * nb; idx += nt) {
      const int li = idx / nb, j = idx % nb, k = j % Ns;
      const float2* s = src + li * M;
      float2 x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < R) x[q] = s[j + q * nb];
      if (Ns > 1) {
#pragma unroll
        for (int q = 1; q < 4; ++q)
          if (q < R) {
            const float2 w = T[(tstep * q * k) % M];
            x[q] = INV ? gcmulc(x[q], w) : gcmul(x[q], w);
          }
      }
      dft_small<INV>(x, R);
      float2* d = dst + li * M + (j / Ns) * Ns * R + k;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < R) d[q * Ns] = x[q];
    }
    __syncthreads();
    float2* tmp = src;
    src = dst;
    dst = tmp;
    Ns *= R;
  }
  if (cols) {
    for (int idx = t; idx < n; idx += nt) {
      const int p = idx / L, li = idx % L;
      base[(size_t)p * M + l0 + li] = src[li * M + p];
    }
  } else {
    for (int idx = t; idx < n; idx += nt) base[(size_t)l0 * M + idx] = src[idx];
  }
}

__device__ __forceinline__ bool window_ok(int2 r, int M, int H, int W) {
  return r.x >= 0 && r.y >= 0 && r.x <= H - M && r.y <= W - M;
}

// wv[i] = P (+ step * dir); invalid windows flag the call and start from 0.
__global__ void k_gm_init(const ChainArgs a, float2* __restrict__ wv, int M) {
  const size_t MM = (size_t)M * M, n = (size_t)a.n_pos * MM;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int il = (int)(idx / MM);
    const int rem = (int)(idx % MM);
    const int2 r = a.pos[a.pos_begin + il];
    float2 p = make_float2(0.f, 0.f);
    if (window_ok(r, M, a.H, a.W)) {
      p = a.probe[rem];
      if (a.probe_dir) {
        const float2 d = a.probe_dir[rem];
        p.x = fmaf(a.probe_step, d.x, p.x);
        p.y = fmaf(a.probe_step, d.y, p.y);
      }
    } else if (rem == 0) {
      *a.status = PTYCHO_ERR_POSITION;
    }
    wv[idx] = p;
  }
}

// Forward transmission of slice s: [store psi_s] then wv *= O_s[window] (+ dir).
// Adjoint (ADJ): store g_phi_s, then wv = conj(O_s[window]) wv; at s = 0 the
// result g_psi_0 goes to the probe-gradient workspace instead.
template <bool ADJ>
__global__ void k_gm_transmit(const ChainArgs a, float2* __restrict__ wv, int M, int s, int store) {
  const size_t MM = (size_t)M * M, n = (size_t)a.n_pos * MM;
  const size_t HW = (size_t)a.H * a.W;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int il = (int)(idx / MM);
    const int rem = (int)(idx % MM);
    const int y = rem / M, x = rem % M;
    const int2 r = a.pos[a.pos_begin + il];
    float2 v = wv[idx];
    if (!window_ok(r, M, a.H, a.W)) {  // skipped window: contributes nothing
      wv[idx] = make_float2(0.f, 0.f);
      if (ADJ && s == 0) __stcs(a.ws_gp + (size_t)il * MM + rem, make_float2(0.f, 0.f));
      continue;
    }
    const size_t oi = (size_t)s * HW + (size_t)(r.x + y) * a.W + (r.y + x);
    if (!ADJ) {
      if (store) __stcs(a.ws_psi + ((size_t)(s - 1) * a.ws_n + il) * MM + rem, v);
      float2 o = a.obj[oi];
      if (a.obj_dir) {
        const float2 d = a.obj_dir[oi];
        o.x = fmaf(a.obj_step, d.x, o.x);
        o.y = fmaf(a.obj_step, d.y, o.y);
      }
      wv[idx] = gcmul(v, o);
    } else {
      __stcs(a.ws_gphi + ((size_t)s * a.ws_n + il) * MM + rem, v);
      const float2 g = gcmulc(v, a.obj[oi]);
      if (s == 0)
        __stcs(a.ws_gp + (size_t)il * MM + rem, g);
      else
        wv[idx] = g;
    }
  }
}

// Spectrum times hs[ky] hs[kx] (the propagator with the 1/M^2 of an
// unnormalised FFT pair folded in), or its conjugate.
template <bool CONJ>
__global__ void k_gm_prop(const ChainArgs a, float2* __restrict__ wv, int M) {
  const size_t MM = (size_t)M * M, n = (size_t)a.n_pos * MM;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int rem = (int)(idx % MM);
    const float2 h = gcmul(a.hs[rem / M], a.hs[rem % M]);
    wv[idx] = CONJ ? gcmulc(wv[idx], h) : gcmul(wv[idx], h);
  }
}

// Far field (unnormalised: M Psi) -> outputs (forward mode) or the residual
// of Eq. 1: loss part per position (FP64, fixed order) and the adjoint seed
// 2 d Psi/|Psi| / M, pre-scaled for the unnormalised inverse.  One block per position.
template <int MODE>
__global__ void __launch_bounds__(256) k_gm_residual(const ChainArgs a, float2* __restrict__ wv, int M) {
  __shared__ double red[8];
  const int il = blockIdx.x, gi = a.pos_begin + il, t = threadIdx.x;
  const size_t MM = (size_t)M * M;
  float2* w = wv + (size_t)il * MM;
  const bool ok = window_ok(a.pos[gi], M, a.H, a.W);
  const float inv_m = 1.0f / (float)M;
  if (MODE == MODE_FORWARD) {
    if (!ok) return;
    for (int k = t; k < (int)MM; k += blockDim.x) {
      const float2 z = make_float2(w[k].x * inv_m, w[k].y * inv_m);
      if (a.psi_out) a.psi_out[(size_t)gi * MM + k] = z;
      if (a.int_out) a.int_out[(size_t)gi * MM + k] = fmaf(z.x, z.x, z.y * z.y);
    }
    return;
  }
  double lsum = 0.0;
  const float* Ii = a.meas + (size_t)gi * MM;
  for (int k = t; k < (int)MM; k += blockDim.x) {
    if (!ok) {
      w[k] = make_float2(0.f, 0.f);
      continue;
    }
    const float2 z = w[k];
    const float A = sqrtf(Ii[k]);
    const float mag = sqrtf(fmaf(z.x, z.x, z.y * z.y));
    const float d = mag * inv_m - A;
    lsum += (double)d * (double)d;
    const float sc = mag > 0.0f ? (2.0f * d) / (mag * (float)M) : 0.0f;
    w[k] = make_float2(z.x * sc, z.y * sc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
  if ((t & 31) == 0) red[t >> 5] = lsum;
  __syncthreads();
  if (t == 0) {
    double tot = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) tot += red[k];
    a.loss_part[il] = ok ? tot : 0.0;
  }
}

int lines_per_block(int M) {
  int best = 1;
  for (int L = 1; L <= M && L * M <= 4096; ++L)
    if (M % L == 0) best = L;
  return best;
}

}  // namespace

bool gm_supported(int M, GmPlan* plan) {
  if (M < 8 || M > 4096) return false;
  GmPlan p{};
  int m = M;
  while (m % 4 == 0) p.r[p.n++] = 4, m /= 4;
  while (m % 2 == 0) p.r[p.n++] = 2, m /= 2;
  while (m % 3 == 0) p.r[p.n++] = 3, m /= 3;
  if (m != 1 || p.n > 16) return false;
  if (plan) *plan = p;
  return true;
}

size_t gm_fft_smem_bytes(int M) { return (2 * (size_t)lines_per_block(M) * M + M) * sizeof(float2); }

// The limit is an attribute of the kernel, shared by every plan in the
// process: always raise it to what the largest supported window needs.
cudaError_t gm_prepare(int) {
  size_t most = 0;
  for (int M = 8; M <= 4096; ++M)
    if (gm_supported(M, nullptr) && gm_fft_smem_bytes(M) > most) most = gm_fft_smem_bytes(M);
  const int bytes = (int)most;
  cudaError_t e = cudaFuncSetAttribute(k_gm_fft<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gm_fft<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

namespace {

struct GmLauncher {
  const ChainArgs& a;
  float2* wv;
  int M;
  GmPlan plan;
  cudaStream_t st;
  int launches = 0;

  unsigned ew_grid() const {
    const size_t n = (size_t)a.n_pos * M * M;
    const size_t b = (n + 255) / 256;
    return (unsigned)(b < 8192 ? b : 8192);
  }
  cudaError_t fft2(bool inv) {
    const int L = lines_per_block(M);
    const unsigned grid = (unsigned)((size_t)a.n_pos * M / L);
    const size_t smem = gm_fft_smem_bytes(M);
    for (int cols = 0; cols < 2; ++cols) {
      if (inv)
        k_gm_fft<true><<<grid, 256, smem, st>>>(wv, M, L, cols, plan, a.tw);
      else
        k_gm_fft<false><<<grid, 256, smem, st>>>(wv, M, L, cols, plan, a.tw);
      ++launches;
    }
    return cudaGetLastError();
  }
  cudaError_t propagate(bool conj) {
    cudaError_t e = fft2(false);
    if (e != cudaSuccess) return e;
    if (conj)
      k_gm_prop<true><<<ew_grid(), 256, 0, st>>>(a, wv, M);
    else
      k_gm_prop<false><<<ew_grid(), 256, 0, st>>>(a, wv, M);
    ++launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return fft2(true);
  }
};

}  // namespace

cudaError_t launch_chain_gm(ChainMode mode, const ChainArgs& a, float2* wv, int M, int* n_launches,
                            cudaStream_t st) {
  if (a.n_pos <= 0) return cudaSuccess;
  GmLauncher g{a, wv, M, GmPlan{}, st};
  if (!gm_supported(M, &g.plan)) return cudaErrorInvalidValue;
  cudaError_t e;
  const bool grad = mode == MODE_GRAD;
  k_gm_init<<<g.ew_grid(), 256, 0, st>>>(a, wv, M);
  ++g.launches;
  for (int s = 0; s < a.S; ++s) {
    k_gm_transmit<false><<<g.ew_grid(), 256, 0, st>>>(a, wv, M, s, grad && s > 0);
    ++g.launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (s < a.S - 1 && (e = g.propagate(false)) != cudaSuccess) return e;
  }
  if ((e = g.fft2(false)) != cudaSuccess) return e;
  switch (mode) {
    case MODE_FORWARD: k_gm_residual<MODE_FORWARD><<<a.n_pos, 256, 0, st>>>(a, wv, M); break;
    case MODE_LOSS: k_gm_residual<MODE_LOSS><<<a.n_pos, 256, 0, st>>>(a, wv, M); break;
    default: k_gm_residual<MODE_GRAD><<<a.n_pos, 256, 0, st>>>(a, wv, M); break;
  }
  ++g.launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (grad) {
    if ((e = g.fft2(true)) != cudaSuccess) return e;
    for (int s = a.S - 1; s >= 0; --s) {
      k_gm_transmit<true><<<g.ew_grid(), 256, 0, st>>>(a, wv, M, s, 1);
      ++g.launches;
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if (s > 0 && (e = g.propagate(true)) != cudaSuccess) return e;
    }
  }
  if (n_launches) *n_launches = g.launches;
  return cudaSuccess;
}

}  // namespace ptycho
