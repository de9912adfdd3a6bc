// Per-position multislice chain: forward model G (Sec. II-B), amplitude
// residual of Eq. 1 and the exact adjoint back to the slices and the probe
// (the per-position term of Eq. 2, Sec. III).
//
// One thread block owns one probe position for its whole slice chain; the
// wave never leaves the SM between slices.  Per slice s the forward pass
// multiplies by the object window O_s[y_i:y_i+M, x_i:x_i+M] (read straight
// from global memory, L2-resident) and, if s < S-1, propagates by
// FFT -> x h -> IFFT.  The exit wave is transformed to the detector; the
// residual gives the loss term and the seed of the adjoint, which runs the
// chain backwards with conjugated factors.
//
// Gradient mode writes, per position, the wave entering every slice s >= 1
// and the gradient w.r.t. every slice's exit wave (streaming stores); the
// object gradient conj(psi_s) * g_phi_s is formed and summed per object tile
// by the deterministic owner-computes reduction in reduce_kernels.cu.
//
// Recompute mode (checkpoint every L slices, K = ceil(S / L) segments) runs
// as K launches so that the workspace does not hold a patch per slice: the
// first (MODE_GRAD_RC) runs the forward model keeping only the checkpoints
// entering segments 1..K-2 and the waves of the last segment, then the
// residual and the adjoint through the last segment, writing its finished
// gradient patches conj(psi_s) g_phi_s over those waves and parking the
// adjoint state.  Each later launch (MODE_RC_SEG, segment j = K-2 .. 0)
// rebuilds segment j's waves from its checkpoint (or the probe) with the
// forward model's exact operations, runs the adjoint through the segment from
// the parked state and parks the state again (segment 0: the probe gradient).
// The host accumulates each segment's patches into the object gradient
// before the next launch overwrites them.
#include "fft2d.cuh"
#include "internal.h"
#include "../../include/ptycho.h"

namespace ptycho {

namespace {

// Elementwise over the pass-0 grouping (natural order), element (py, px).
template <class C, class F>
__device__ __forceinline__ void for_p0(int t, F&& f) {
  using P = PassShape<C, 0>;
  t = opaque(t);
  static_for<0, P::Q>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    int py0, px0;
    C::template base<0>(t, q, py0, px0);
    static_for<0, P::RY>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      static_for<0, P::RX>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        f(q * P::G + a * P::RX + b, py0 + a * P::SY, px0 + b * P::SX);
      });
    });
  });
}

// Elementwise over the pass-2 grouping (spectrum), frequency (ky, kx).
template <class C, class F>
__device__ __forceinline__ void for_p2(int t, F&& f) {
  using P = PassShape<C, 2>;
  t = opaque(t);
  static_for<0, P::Q>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    int py, px;
    C::template base<2>(t, q, py, px);
    const int ky0 = freq_y<C>(py), kx0 = freq_x<C>(px);
    static_for<0, P::RY>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      static_for<0, P::RX>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        f(q * P::G + a * P::RX + b, ky0 + C::ry(0) * C::ry(1) * a, kx0 + C::rx(0) * C::rx(1) * b);
      });
    });
  });
}

__device__ __forceinline__ float2 ldg2(const float2* p) { return __ldg(p); }

// The forward model's propagations multiply by the full propagator table
// (one rounding per element fewer; the residual amplifies the forward
// model's rounding), the adjoint's by the separable factors in shared memory.
#ifndef PTYCHO_PROP_TABLE
#define PTYCHO_PROP_TABLE 1
#endif
template <class C>
__device__ __forceinline__ void mul_prop_fwd(float2 (&v)[C::V], const float2* hs, const float2* h2, int t) {
#if PTYCHO_PROP_TABLE
  mul_table<C, false>(v, h2, t);
#else
  mul_separable<C, false>(v, hs, t);
#endif
}

// Recompute mode's finished patches are read once by the accumulation that
// follows each launch: streaming stores by default; plain stores (to keep a
// chunk's patches in L2 when the chunk is small enough) with
// PTYCHO_PATCH_STORE_CS=0.
#ifndef PTYCHO_PATCH_STORE_CS
#define PTYCHO_PATCH_STORE_CS 1
#endif
__device__ __forceinline__ void store_patch(float2* p, float2 v) {
#if PTYCHO_PATCH_STORE_CS
  __stcs(p, v);
#else
  *p = v;
#endif
}

}  // namespace

template <int M, int MODE>
__global__ void __launch_bounds__(Cfg<M>::T, Cfg<M>::MIN_BLOCKS) k_chain(const ChainArgs a) {
  using C = Cfg<M>;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* tw = sm + M * M;
  float2* hs = tw + M;
  double* red = reinterpret_cast<double*>(hs + M);
  const int t = threadIdx.x;
  const int il = blockIdx.x;
  const int gi = a.pos_begin + il;

  for (int k = t; k < M; k += C::T) {
    tw[k] = a.tw[k];
    hs[k] = a.hs[k];
  }
  const int2 r = a.pos[gi];
  const int yi = r.x, xi = r.y;
  if (yi < 0 || xi < 0 || yi > a.H - M || xi > a.W - M) {
    // Window outside the object: contribute nothing, flag the call.  (The
    // accumulation skips such windows, so no patch needs clearing.)
    if (t == 0 && MODE != MODE_RC_SEG) {
      *a.status = PTYCHO_ERR_POSITION;
      if (MODE != MODE_FORWARD) a.loss_part[il] = 0.0;
    }
    if (MODE == MODE_GRAD || MODE == MODE_GRAD_RC || (MODE == MODE_RC_SEG && a.seg == 0))
      for (int k = t; k < M * M; k += C::T) a.ws_gp[(size_t)il * M * M + k] = make_float2(0.f, 0.f);
    return;
  }
  __syncthreads();

  const size_t MM = (size_t)M * M;
  const size_t HW = (size_t)a.H * a.W;
  const float2* objw = a.obj + (size_t)yi * a.W + xi;
  // (gradient mode always evaluates at obj itself)
  constexpr bool GRAD = MODE == MODE_GRAD || MODE == MODE_GRAD_RC;
  const float2* dirw = (!GRAD && a.obj_dir) ? a.obj_dir + (size_t)yi * a.W + xi : nullptr;
  const int L = (MODE == MODE_GRAD_RC || MODE == MODE_RC_SEG) ? a.ckpt_L : 1;
  const int K = (a.S + L - 1) / L;  // segments (recompute mode)
  // Recompute-mode slots of ws_psi (each [ws_n][M][M]): checkpoints entering
  // segments 1..K-2 at 0..K-3, the L waves (then patches) of the segment being
  // differentiated from K-2, the parked adjoint state at K-2+L.
  auto rc_slot = [&](int slot) { return a.ws_psi + ((size_t)slot * a.ws_n + il) * MM; };
  const int seg_slot = K - 2, park_slot = K - 2 + L;

  float2 v[C::V];
  if constexpr (MODE == MODE_RC_SEG) {
    // Segment j of the adjoint with recomputation (j <= K-2, so s1 = s0 + L).
    const int j = a.seg, s0 = j * L, s1 = s0 + L;
    if (j == 0) {
      for_p0<C>(t, [&](int e, int py, int px) { v[e] = ldg2(a.probe + py * M + px); });
    } else {
      const float2* ck = rc_slot(j - 1);
      for_p0<C>(t, [&](int e, int py, int px) { v[e] = __ldcs(ck + py * M + px); });
    }
    for (int s = s0; s < s1; ++s) {
      float2* seg = rc_slot(seg_slot + (s - s0));
      for_p0<C>(t, [&](int e, int py, int px) { seg[py * M + px] = v[e]; });
      if (s < s1 - 1) {
        const float2* ow = objw + (size_t)s * HW;
        for_p0<C>(t, [&](int e, int py, int px) { v[e] = cmul(v[e], ldg2(ow + (size_t)py * a.W + px)); });
        fft_fwd<C>(v, sm, tw, t);
        mul_prop_fwd<C>(v, hs, a.h2, t);
        fft_inv<C>(v, sm, tw, t);
      }
    }
    const float2* park = rc_slot(park_slot);  // written by this thread: coherent loads
    for_p0<C>(t, [&](int e, int py, int px) { v[e] = park[py * M + px]; });
    for (int s = s1 - 1; s >= s0; --s) {
      float2* seg = rc_slot(seg_slot + (s - s0));
      for_p0<C>(t, [&](int e, int py, int px) {
        const int k = py * M + px;
        store_patch(seg + k, cconjmul(seg[k], v[e]));  // conj(psi_s) g_phi_s over psi_s
      });
      const float2* ow = objw + (size_t)s * HW;
      for_p0<C>(t, [&](int e, int py, int px) { v[e] = cmulc(v[e], ldg2(ow + (size_t)py * a.W + px)); });
      if (s > 0) {
        fft_fwd<C, true>(v, sm, tw, t);
        mul_separable<C, true>(v, hs, t);
        fft_inv<C, true>(v, sm, tw, t);
      }
    }
    float2* out = j > 0 ? rc_slot(park_slot) : a.ws_gp + (size_t)il * MM;
    for_p0<C>(t, [&](int e, int py, int px) { out[py * M + px] = v[e]; });
    return;
  }
  // psi_0 = P
  for_p0<C>(t, [&](int e, int py, int px) {
    float2 p = ldg2(a.probe + py * M + px);
    if (a.probe_dir) {
      const float2 d = ldg2(a.probe_dir + py * M + px);
      p.x = fmaf(a.probe_step, d.x, p.x);
      p.y = fmaf(a.probe_step, d.y, p.y);
    }
    v[e] = p;
  });

  for (int s = 0; s < a.S; ++s) {
    if (MODE == MODE_GRAD && s > 0) {
      float2* dst = a.ws_psi + ((size_t)(s - 1) * a.ws_n + il) * MM;
      for_p0<C>(t, [&](int e, int py, int px) { __stcs(dst + py * M + px, v[e]); });
    }
    if (MODE == MODE_GRAD_RC && s > 0 && s % L == 0 && s / L <= K - 2) {  // checkpoint entering segment s / L
      float2* dst = rc_slot(s / L - 1);
      for_p0<C>(t, [&](int e, int py, int px) { __stcs(dst + py * M + px, v[e]); });
    }
    if (MODE == MODE_GRAD_RC && s >= (K - 1) * L) {  // the last segment's waves
      float2* dst = rc_slot(seg_slot + (s - (K - 1) * L));
      for_p0<C>(t, [&](int e, int py, int px) { dst[py * M + px] = v[e]; });
    }
    // phi_s = psi_s * O_s[window]  (O + step * dir during a line search)
    const float2* ow = objw + (size_t)s * HW;
    const float2* dw = dirw ? dirw + (size_t)s * HW : nullptr;
    for_p0<C>(t, [&](int e, int py, int px) {
      float2 o = ldg2(ow + (size_t)py * a.W + px);
      if (dw) {
        const float2 d = ldg2(dw + (size_t)py * a.W + px);
        o.x = fmaf(a.obj_step, d.x, o.x);
        o.y = fmaf(a.obj_step, d.y, o.y);
      }
      v[e] = cmul(v[e], o);
    });
    if (s < a.S - 1) {
      fft_fwd<C>(v, sm, tw, t);
      mul_prop_fwd<C>(v, hs, a.h2, t);
      fft_inv<C>(v, sm, tw, t);
    }
  }
  fft_fwd<C>(v, sm, tw, t);  // far field times M (unnormalised)

  const float inv_m = 1.0f / (float)M;
  if constexpr (MODE == MODE_FORWARD) {
    float2* po = a.psi_out ? a.psi_out + (size_t)gi * MM : nullptr;
    float* io = a.int_out ? a.int_out + (size_t)gi * MM : nullptr;
    for_p2<C>(t, [&](int e, int ky, int kx) {
      const float2 z = make_float2(v[e].x * inv_m, v[e].y * inv_m);
      if (po) po[ky * M + kx] = z;
      if (io) io[ky * M + kx] = fmaf(z.x, z.x, z.y * z.y);
    });
    return;
  } else {
    // Amplitude residual (Eq. 1): d = |Psi| - sqrt(I); loss term d^2, summed
    // in FP64.  Seed of the adjoint g_Psi = 2 d Psi/|Psi| (0 where Psi = 0),
    // pre-scaled by 1/M so the unnormalised inverse gives F^H g_Psi.
    const float* Ii = a.meas + (size_t)gi * MM;
    double lsum = 0.0;
    for_p2<C>(t, [&](int e, int ky, int kx) {
      const float2 z = v[e];
      const float A = sqrtf(__ldg(Ii + ky * M + kx));
      const float mag = sqrtf(fmaf(z.x, z.x, z.y * z.y));  // |M Psi|
      const float d = mag * inv_m - A;
      lsum += (double)d * (double)d;
      const float sc = mag > 0.0f ? (2.0f * d) / (mag * (float)M) : 0.0f;
      v[e] = make_float2(z.x * sc, z.y * sc);
    });
    // block reduction in a fixed order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
    if ((t & 31) == 0) red[t >> 5] = lsum;
    __syncthreads();
    if (t == 0) {
      double tot = 0.0;
      for (int w = 0; w < C::T / 32; ++w) tot += red[w];
      a.loss_part[il] = tot;
    }
    if constexpr (MODE == MODE_LOSS) {
      return;
    } else if constexpr (MODE == MODE_GRAD) {
      fft_inv<C, true>(v, sm, tw, t);  // g_phi for the last slice
      for (int s = a.S - 1; s >= 0; --s) {
        float2* dst = a.ws_gphi + ((size_t)s * a.ws_n + il) * MM;
        for_p0<C>(t, [&](int e, int py, int px) { __stcs(dst + py * M + px, v[e]); });
        const float2* ow = objw + (size_t)s * HW;
        for_p0<C>(t, [&](int e, int py, int px) {
          v[e] = cmulc(v[e], ldg2(ow + (size_t)py * a.W + px));  // g_psi = conj(O) g_phi
        });
        if (s > 0) {
          fft_fwd<C, true>(v, sm, tw, t);
          mul_separable<C, true>(v, hs, t);
          fft_inv<C, true>(v, sm, tw, t);
        }
      }
    } else {
      // Recompute mode, first launch: the adjoint through the last segment
      // [s0, S), whose waves the forward kept, then park the state for the
      // launch of segment K-2.
      fft_inv<C, true>(v, sm, tw, t);
      const int s0 = (K - 1) * L;
      for (int s = a.S - 1; s >= s0; --s) {
        float2* seg = rc_slot(seg_slot + (s - s0));
        for_p0<C>(t, [&](int e, int py, int px) {
          const int k = py * M + px;
          store_patch(seg + k, cconjmul(seg[k], v[e]));  // conj(psi_s) g_phi_s over psi_s
        });
        const float2* ow = objw + (size_t)s * HW;
        for_p0<C>(t, [&](int e, int py, int px) { v[e] = cmulc(v[e], ldg2(ow + (size_t)py * a.W + px)); });
        fft_fwd<C, true>(v, sm, tw, t);  // s >= s0 >= L >= 1
        mul_separable<C, true>(v, hs, t);
        fft_inv<C, true>(v, sm, tw, t);
      }
      float2* park = rc_slot(park_slot);
      for_p0<C>(t, [&](int e, int py, int px) { park[py * M + px] = v[e]; });
      return;
    }
    if constexpr (MODE == MODE_GRAD) {
      float2* gp = a.ws_gp + (size_t)il * MM;
      for_p0<C>(t, [&](int e, int py, int px) { __stcs(gp + py * M + px, v[e]); });
    }
  }
}

int chain_threads(int M) { return M == 128 ? Cfg<128>::T : Cfg<64>::T; }

size_t chain_smem_bytes(int M) {
  return (size_t)M * M * sizeof(float2) + 2 * (size_t)M * sizeof(float2) +
         (size_t)(chain_threads(M) / 32) * sizeof(double);
}

template <int M>
static cudaError_t prepare_m() {
  const int bytes = (int)chain_smem_bytes(M);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_chain<M, MODE_FORWARD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_chain<M, MODE_LOSS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_chain<M, MODE_GRAD_RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_chain<M, MODE_RC_SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_chain<M, MODE_GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t chain_prepare(int M) { return M == 128 ? prepare_m<128>() : prepare_m<64>(); }

int chain_blocks_per_sm(int M) {
  int n = 0;
  const cudaError_t e =
      M == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_chain<128, MODE_GRAD>, Cfg<128>::T,
                                                               chain_smem_bytes(128))
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_chain<64, MODE_GRAD>, Cfg<64>::T,
                                                               chain_smem_bytes(64));
  return e == cudaSuccess ? n : 0;
}

template <int M>
static cudaError_t launch_m(ChainMode mode, const ChainArgs& a, cudaStream_t st) {
  const dim3 grid(a.n_pos), block(Cfg<M>::T);
  const size_t smem = chain_smem_bytes(M);
  switch (mode) {
    case MODE_FORWARD: k_chain<M, MODE_FORWARD><<<grid, block, smem, st>>>(a); break;
    case MODE_LOSS: k_chain<M, MODE_LOSS><<<grid, block, smem, st>>>(a); break;
    case MODE_GRAD_RC: k_chain<M, MODE_GRAD_RC><<<grid, block, smem, st>>>(a); break;
    case MODE_RC_SEG: k_chain<M, MODE_RC_SEG><<<grid, block, smem, st>>>(a); break;
    default: k_chain<M, MODE_GRAD><<<grid, block, smem, st>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_chain(int M, ChainMode mode, const ChainArgs& a, cudaStream_t st) {
  if (a.n_pos <= 0) return cudaSuccess;
  return M == 128 ? launch_m<128>(mode, a, st) : launch_m<64>(mode, a, st);
}

}  // namespace ptycho
