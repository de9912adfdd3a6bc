// Generic-window slice chain: any probe window M = 2^a 3^b (8 <= M <= 4096)
// that the register-resident kernels do not cover (they take M = 64, 128).
//
// The chunk's positions advance through the multislice model (Sec. II-B)
// together, slice by slice: their waves live in a global buffer wv[n][M][M].
// Every pass loads a block of rows or columns of one wave into shared memory,
// transforms them with mixed-radix (8/4/2/3) Stockham stages in natural
// order, and writes them back.  Because the Fresnel factor is separable, a
// propagation is a row pass and a column pass, each running FFT, factor and
// inverse on its lines; the transmission of a slice and its adjoint ride on
// the row passes.  The amplitude residual of Eq. 1 is one pointwise kernel.
// The workspace it fills (entering waves, exit-wave gradients, probe-gradient
// parts, loss parts) has the layout of the register-resident kernels, so the
// tiled reductions are shared.
#include "../../include/ptycho.h"
#include "fft2d.cuh"
#include "internal.h"

namespace ptycho {

namespace {

// Small DFT of a register array in natural order, forward kernel
// exp(-2 pi i n k / R), inverse its conjugate, unnormalised.
template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2 (&x)[R]) {
  if constexpr (R == 2) {
    dft2(x[0], x[1]);
  } else if constexpr (R == 3) {
    // X1 = t2 -+ i s3 (b - c), X2 = t2 +- i s3 (b - c), t2 = a - (b + c)/2
    const float s3 = 0.86602540378443864676f;
    const float2 a = x[0], b = x[1], c = x[2];
    const float2 t1 = cadd(b, c);
    const float2 t2 = make_float2(fmaf(-0.5f, t1.x, a.x), fmaf(-0.5f, t1.y, a.y));
    const float2 d = make_float2(s3 * (b.x - c.x), s3 * (b.y - c.y));
    const float2 mid = mul_mi<INV>(d);
    x[0] = cadd(a, t1);
    x[1] = cadd(t2, mid);
    x[2] = csub(t2, mid);
  } else if constexpr (R == 4) {
    dft4<INV>(x[0], x[1], x[2], x[3]);
  } else {
    static_assert(R == 8, "radix 2, 3, 4 or 8");
    dft8<INV>(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7]);
  }
}

// Shared-memory slot of element i of a line: one padding slot every 16
// elements, which spreads the radix-8 first stage (outputs 8 apart across
// threads) over the banks; the odd line stride does the same for the column
// transposes.  (Simulated bank wavefronts per warp access, ideal 2: 2.0-2.8
// for M = 96, 192, 256 against 3.3-4.7 unpadded.)
__host__ __device__ constexpr int gm_pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int gm_line_stride(int M) { return M + M / 16 + 1; }

// One Stockham autosort stage of radix R on L lines of length M (line
// stride LS in shared memory, padded slots), after spans of Ns: butterfly j takes
// x[j + q M/R], twiddles it by w_{Ns R}^{q (j mod Ns)} = w_M^{tstep q k}, and
// writes y[(j - k) R + k + q Ns].  tstep q k < M, so the table needs no wrap.
template <int R, bool INV>
__device__ __forceinline__ void gm_stage(const float2* __restrict__ src, float2* __restrict__ dst, int M, int LS,
                                         int L, int Ns, const float2* __restrict__ T, int t, int nt) {
  const int nb = M / R;
  const int tstep = M / (Ns * R);
  for (int idx = t; idx < L * nb; idx += nt) {
    const int li = idx / nb;
    const int j = idx - li * nb;
    const int k = j % Ns;
    const float2* s = src + li * LS;
    float2 x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = s[gm_pad(j + q * nb)];
    if (Ns > 1) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const float2 w = T[tstep * q * k];
        x[q] = INV ? cmulc(x[q], w) : cmul(x[q], w);
      }
    }
    dft_r<R, INV>(x);
    float2* d = dst + li * LS;
    const int d0 = (j - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) d[gm_pad(d0 + q * Ns)] = x[q];
  }
}

// Radix schedule of a window: as many 8s as divide it, then 4, 2, then 3s.
__host__ __device__ constexpr int gm_radix_at(int M, int i) {
  int m = M, k = 0;
  const int order[4] = {8, 4, 2, 3};
  for (int o = 0; o < 4; ++o)
    while (m % order[o] == 0 && m > 1) {
      if (k == i) return order[o];
      m /= order[o];
      ++k;
    }
  return 0;
}
__host__ __device__ constexpr int gm_n_stages(int M) {
  int n = 0;
  while (gm_radix_at(M, n) != 0) ++n;
  return n;
}
// Lines per block: the largest divisor of M with L M <= 4096.
__host__ __device__ constexpr int gm_lines(int M) {
  int best = 1;
  for (int L = 1; L <= M && L * M <= 4096; ++L)
    if (M % L == 0) best = L;
  return best;
}

// Stages with everything known at compile time (window MC): index
// arithmetic folds to multiplies and shifts.
template <bool INV, int MC, int I, int NS>
__device__ __forceinline__ float2* gm_stages_ct(float2* src, float2* dst, const float2* T, int t) {
  if constexpr (I == gm_n_stages(MC)) {
    return src;
  } else {
    constexpr int R = gm_radix_at(MC, I);
    gm_stage<R, INV>(src, dst, MC, gm_line_stride(MC), gm_lines(MC), NS, T, t, 256);
    __syncthreads();
    return gm_stages_ct<INV, MC, I + 1, NS * R>(dst, src, T, t);
  }
}

// All stages of one transform of the block's lines; returns the buffer that
// holds the result.  MC = 0: the radix schedule is read from the plan.
template <bool INV, int MC>
__device__ __forceinline__ float2* gm_transform(float2* src, float2* dst, int M, int L, const GmPlan& plan,
                                                const float2* T, int t) {
  if constexpr (MC > 0) {
    return gm_stages_ct<INV, MC, 0, 1>(src, dst, T, t);
  } else {
    int Ns = 1;
    for (int st = 0; st < plan.n; ++st) {
      const int R = plan.r[st];
      if (R == 8)
        gm_stage<8, INV>(src, dst, M, gm_line_stride(M), L, Ns, T, t, 256);
      else if (R == 4)
        gm_stage<4, INV>(src, dst, M, gm_line_stride(M), L, Ns, T, t, 256);
      else if (R == 2)
        gm_stage<2, INV>(src, dst, M, gm_line_stride(M), L, Ns, T, t, 256);
      else
        gm_stage<3, INV>(src, dst, M, gm_line_stride(M), L, Ns, T, t, 256);
      __syncthreads();
      float2* tmp = src;
      src = dst;
      dst = tmp;
      Ns *= R;
    }
    return src;
  }
}

__device__ __forceinline__ bool window_ok(int2 r, int M, int H, int W) {
  return r.x >= 0 && r.y >= 0 && r.x <= H - M && r.y <= W - M;
}

// What one line pass does between loading and storing its lines.
enum : int { GM_FFT = 0, GM_IFFT = 1, GM_PROP = 2, GM_PROP_CONJ = 3 };

struct GmLineArgs {
  int op;     // GM_*: transform, inverse, or 1-D propagation (FFT, x hs[k], IFFT)
  int cols;   // 0: the lines are rows, 1: columns
  int s;      // slice of a fused transmission (row passes only)
  int pre;    // forward transmission on load: [store psi_s], times O_s[window]
  int post;   // adjoint transmission on store: store g_phi_s, times conj(O_s[window])
  int store;  // with pre: keep psi_s in the workspace
};

// One pass over L rows or columns of each wave.  The Fresnel factor is
// separable, h(ky, kx) = h1(ky) h1(kx), so a propagation F^-1 h F is a 1-D
// propagation of every row followed by one of every column: each pass keeps
// its lines in shared memory through FFT, the factor hs[k] = h1(k)/M and the
// inverse.  Row passes also apply the slice's transmission (Sec. II-B) on
// load, or its adjoint on store, so a slice costs one row and one column
// pass each way.
//   forward transmission (pre):  psi_0 = P (+ step dir); [psi_s -> workspace];
//                                v = psi_s O_s[window] (+ step dir)
//   adjoint transmission (post): g_phi_s -> workspace, v = conj(O_s[window]) g_phi_s,
//                                at s = 0 into the probe-gradient workspace instead.
// Skipped (out-of-range) windows carry zeros and flag the call.
template <int MC>
__global__ void __launch_bounds__(256) k_gm_line(const ChainArgs a, float2* __restrict__ wv, int M, GmPlan plan,
                                                 GmLineArgs g) {
  if constexpr (MC > 0) M = MC;
  const int L = MC > 0 ? gm_lines(MC) : gm_lines(M);
  const int LS = gm_line_stride(M);
  extern __shared__ float2 gsm[];
  float2* A = gsm;
  float2* B = A + (size_t)L * LS;
  float2* T = B + (size_t)L * LS;
  float2* Hs = T + M;
  const int t = threadIdx.x;
  for (int k = t; k < M; k += 256) {
    T[k] = a.tw[k];
    Hs[k] = a.hs[k];
  }
  const size_t MM = (size_t)M * M;
  const int g0 = blockIdx.x * L;  // first line of this block (L divides M)
  const int il = g0 / M;
  const int l0 = g0 - il * M;
  float2* base = wv + (size_t)il * MM;
  const int2 r = a.pos[a.pos_begin + il];
  const bool ok = window_ok(r, M, a.H, a.W);
  const size_t HW = (size_t)a.H * a.W;
  const int n = L * M;
  // Loads are issued in batches of U per thread before their results are
  // used, so each thread keeps U global reads in flight.
  constexpr int U = 8;
  if (g.cols) {
    for (int i0 = 0; i0 < n; i0 += 256 * U) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = i0 + u * 256 + t;
        if (idx < n) {
          const int p = idx / L, li = idx - p * L;
          v[u] = base[(size_t)p * M + l0 + li];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = i0 + u * 256 + t;
        if (idx < n) {
          const int p = idx / L, li = idx - p * L;
          A[li * LS + gm_pad(p)] = v[u];
        }
      }
    }
  } else {
    // Row pass with the forward transmission: the wave entering slice s is
    // the probe at s = 0 (P + step dir on a line-search trial), else wv.
    const bool from_probe = g.pre && g.s == 0;
    const float2* src = from_probe ? a.probe : base + (size_t)l0 * M;
    if (from_probe) src += (size_t)l0 * M;
    if (g.pre && !ok && l0 == 0 && t == 0) *a.status = PTYCHO_ERR_POSITION;
    for (int i0 = 0; i0 < n; i0 += 256 * U) {
      float2 v[U], o[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = i0 + u * 256 + t;
        if (idx < n) {
          v[u] = src[idx];
          if (g.pre && ok) {
            const int li = idx / M, x = idx - li * M;
            const size_t oi = (size_t)g.s * HW + (size_t)(r.x + l0 + li) * a.W + (r.y + x);
            o[u] = a.obj[oi];
            if (a.obj_dir) {
              const float2 d = a.obj_dir[oi];
              o[u].x = fmaf(a.obj_step, d.x, o[u].x);
              o[u].y = fmaf(a.obj_step, d.y, o[u].y);
            }
            if (from_probe && a.probe_dir) {
              const float2 d = a.probe_dir[(size_t)l0 * M + idx];
              v[u].x = fmaf(a.probe_step, d.x, v[u].x);
              v[u].y = fmaf(a.probe_step, d.y, v[u].y);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = i0 + u * 256 + t;
        if (idx < n) {
          const int li = idx / M, x = idx - li * M;
          float2 w = v[u];
          if (g.pre) {
            if (!ok) {
              w = make_float2(0.f, 0.f);
            } else {
              if (g.store) __stcs(a.ws_psi + ((size_t)(g.s - 1) * a.ws_n + il) * MM + (size_t)l0 * M + idx, w);
              w = cmul(w, o[u]);
            }
          }
          A[li * LS + gm_pad(x)] = w;
        }
      }
    }
  }
  __syncthreads();
  float2* out;
  if (g.op == GM_FFT) {
    out = gm_transform<false, MC>(A, B, M, L, plan, T, t);
  } else if (g.op == GM_IFFT) {
    out = gm_transform<true, MC>(A, B, M, L, plan, T, t);
  } else {
    float2* mid = gm_transform<false, MC>(A, B, M, L, plan, T, t);
    const bool cj = g.op == GM_PROP_CONJ;
    for (int idx = t; idx < n; idx += 256) {
      const int li = idx / M, k = idx - li * M;
      float2& z = mid[li * LS + gm_pad(k)];
      z = cj ? cmulc(z, Hs[k]) : cmul(z, Hs[k]);
    }
    __syncthreads();
    out = gm_transform<true, MC>(mid, mid == A ? B : A, M, L, plan, T, t);
  }
  if (g.cols) {
    for (int idx = t; idx < n; idx += 256) {
      const int p = idx / L, li = idx - p * L;
      base[(size_t)p * M + l0 + li] = out[li * LS + gm_pad(p)];
    }
  } else if (!g.post) {
    for (int idx = t; idx < n; idx += 256) {
      const int li = idx / M, x = idx - li * M;
      base[(size_t)l0 * M + idx] = out[li * LS + gm_pad(x)];
    }
  } else if (!ok) {
    for (int idx = t; idx < n; idx += 256) {
      const size_t rem = (size_t)l0 * M + idx;
      base[rem] = make_float2(0.f, 0.f);
      if (g.s == 0) __stcs(a.ws_gp + (size_t)il * MM + rem, make_float2(0.f, 0.f));
    }
  } else {
    for (int i0 = 0; i0 < n; i0 += 256 * U) {
      float2 o[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = i0 + u * 256 + t;
        if (idx < n) {
          const int li = idx / M, x = idx - li * M;
          o[u] = a.obj[(size_t)g.s * HW + (size_t)(r.x + l0 + li) * a.W + (r.y + x)];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = i0 + u * 256 + t;
        if (idx < n) {
          const int li = idx / M, x = idx - li * M;
          const size_t rem = (size_t)l0 * M + idx;
          const float2 v = out[li * LS + gm_pad(x)];
          __stcs(a.ws_gphi + ((size_t)g.s * a.ws_n + il) * MM + rem, v);
          const float2 gv = cmulc(v, o[u]);
          if (g.s == 0)
            __stcs(a.ws_gp + (size_t)il * MM + rem, gv);
          else
            base[rem] = gv;
        }
      }
    }
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

}  // namespace

bool gm_supported(int M, GmPlan* plan) {
  if (M < 8 || M > 4096) return false;
  GmPlan p{};
  p.n = gm_n_stages(M);
  if (p.n > 16) return false;
  int prod = 1;
  for (int i = 0; i < p.n; ++i) prod *= (p.r[i] = gm_radix_at(M, i));
  if (prod != M) return false;
  if (plan) *plan = p;
  return true;
}

size_t gm_fft_smem_bytes(int M) {
  return (2 * (size_t)gm_lines(M) * gm_line_stride(M) + 2 * (size_t)M) * sizeof(float2);
}

namespace {

// Windows with a compile-time instance of the line pass; others take the
// runtime radix schedule.
template <int MC>
cudaError_t gm_set_smem(int bytes) {
  return cudaFuncSetAttribute(k_gm_line<MC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

// The limit is an attribute of the kernel, shared by every plan in the
// process: always raise it to what the largest window it serves needs.
cudaError_t gm_prepare(int) {
  size_t most = 0;
  for (int M = 8; M <= 4096; ++M)
    if (gm_supported(M, nullptr) && gm_fft_smem_bytes(M) > most) most = gm_fft_smem_bytes(M);
  cudaError_t e;
  if ((e = gm_set_smem<0>((int)most)) != cudaSuccess) return e;
  if ((e = gm_set_smem<96>((int)gm_fft_smem_bytes(96))) != cudaSuccess) return e;
  if ((e = gm_set_smem<192>((int)gm_fft_smem_bytes(192))) != cudaSuccess) return e;
  return gm_set_smem<256>((int)gm_fft_smem_bytes(256));
}

namespace {

struct GmLauncher {
  const ChainArgs& a;
  float2* wv;
  int M;
  GmPlan plan;
  cudaStream_t st;
  int launches = 0;

  cudaError_t line(int op, int cols, int s = 0, int pre = 0, int post = 0, int store = 0) {
    const GmLineArgs g{op, cols, s, pre, post, store};
    const unsigned grid = (unsigned)((size_t)a.n_pos * M / gm_lines(M));
    const size_t smem = gm_fft_smem_bytes(M);
    switch (M) {
      case 96: k_gm_line<96><<<grid, 256, smem, st>>>(a, wv, M, plan, g); break;
      case 192: k_gm_line<192><<<grid, 256, smem, st>>>(a, wv, M, plan, g); break;
      case 256: k_gm_line<256><<<grid, 256, smem, st>>>(a, wv, M, plan, g); break;
      default: k_gm_line<0><<<grid, 256, smem, st>>>(a, wv, M, plan, g); break;
    }
    ++launches;
    return cudaGetLastError();
  }
};

}  // namespace

// Forward: for each slice s < S-1 one row pass (transmission, propagation
// along x) and one column pass (propagation along y); the last slice's row
// and column passes are the far-field transform.  Adjoint, in reverse: the
// inverse far field (column pass, then row pass ending in the adjoint
// transmission of slice S-1), then per slice a conjugate-propagation column
// pass and a row pass ending in the adjoint transmission.
cudaError_t launch_chain_gm(ChainMode mode, const ChainArgs& a, float2* wv, int M, int* n_launches,
                            cudaStream_t st) {
  if (a.n_pos <= 0) return cudaSuccess;
  GmLauncher g{a, wv, M, GmPlan{}, st};
  if (!gm_supported(M, &g.plan)) return cudaErrorInvalidValue;
  cudaError_t e;
  const bool grad = mode == MODE_GRAD;
  for (int s = 0; s < a.S; ++s) {
    const bool last = s == a.S - 1;
    const int op = last ? GM_FFT : GM_PROP;
    if ((e = g.line(op, 0, s, 1, 0, grad && s > 0)) != cudaSuccess) return e;
    if ((e = g.line(op, 1)) != cudaSuccess) return e;
  }
  switch (mode) {
    case MODE_FORWARD: k_gm_residual<MODE_FORWARD><<<a.n_pos, 256, 0, st>>>(a, wv, M); break;
    case MODE_LOSS: k_gm_residual<MODE_LOSS><<<a.n_pos, 256, 0, st>>>(a, wv, M); break;
    default: k_gm_residual<MODE_GRAD><<<a.n_pos, 256, 0, st>>>(a, wv, M); break;
  }
  ++g.launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (grad) {
    for (int s = a.S - 1; s >= 0; --s) {
      const int op = s == a.S - 1 ? GM_IFFT : GM_PROP_CONJ;
      if ((e = g.line(op, 1)) != cudaSuccess) return e;
      if ((e = g.line(op, 0, s, 0, 1)) != cudaSuccess) return e;
    }
  }
  if (n_launches) *n_launches = g.launches;
  return cudaSuccess;
}

}  // namespace ptycho
