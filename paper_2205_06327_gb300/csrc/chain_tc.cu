// Per-position multislice chain with the 2-D transforms done as BF16 hi/lo
// split DFT matrix products on the tensor cores (tcgen05, FP32 accumulation in
// tensor memory).  Same inputs, outputs and workspace as the FP32 kernel in
// chain_kernels.cu, so the tiled reductions are shared.
//
// Every transform of the chain is a "sandwich" X -> C X C with a symmetric
// complex 128 x 128 matrix C: the Fresnel step (Sec. II-B) is separable,
// F^-1 diag(h(ky) h(kx)) F = K_y (.) K_x with K = F^-1 diag(h_1) F, and the
// far field is the orthonormal DFT matrix F on both sides.  The adjoint uses
// conj(C) (the sign of Im C flips).  With D = A * B on the tensor core:
//   stage 1: D1 = C * W          (A = C from tensor memory, B = W)
//   stage 2: D2 = C * D1^T = (C W C)^T
// One thread owns one tensor-memory lane, so after stage 2 thread j holds
// column j of the result; keeping the wave column-held makes both B operands
// K-major rows that each thread writes contiguously.
//
// Precision: every operand is split x = x_hi + x_lo in BF16 (or in IEEE half,
// F16 = true: 22 significant bits instead of 16, same tensor rate, |x| <
// 65504) and each real product uses A_hi B_hi + A_hi B_lo + A_lo B_hi;
// complex products use four real ones.  Pointwise work (transmission,
// residual) stays FP32, the loss sum FP64.
//
// 512 threads (or 256): warp w owns tensor-memory lanes 32 (w % 4) .. + 31
// (one row m of the accumulator per thread) and column group w / 4.
#include "../../include/ptycho.h"
#include "internal.h"
#include "tc_bf16.cuh"

namespace ptycho {

namespace {

constexpr int TM = 128;                 // window (tensor tile) size
constexpr int kPlaneBytes = TM * TM * 2;  // one BF16 plane
constexpr uint32_t kColD = 0;             // D_re at columns [0,128), D_im at [128,256)
constexpr uint32_t kColA = 256;           // A planes: re_hi, re_lo, im_hi, im_lo, 64 columns each
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at the maximum SM clock
// Threads per block: 128 x (column groups).  Thread t owns tensor-memory lane
// t % 128 and column group t / 128 (8 / groups chunks of 16 columns).
#ifndef PTYCHO_TC_THREADS
#define PTYCHO_TC_THREADS 512
#endif
constexpr int kTcThreads = PTYCHO_TC_THREADS;
constexpr int kTcGroups = kTcThreads / 128;
constexpr int kTcChunks = 8 / kTcGroups;  // 16-column chunks per thread
static_assert(kTcThreads == 256 || kTcThreads == 512, "256 or 512 threads");

__device__ __forceinline__ float2 cmul_tc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc_tc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// Terms (A plane, B plane, Im(C) term) of D_re and D_im: planes 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo.
__constant__ int c_terms_re[6][3] = {{0, 0, 0}, {0, 1, 0}, {1, 0, 0}, {2, 2, 1}, {2, 3, 1}, {3, 2, 1}};
__constant__ int c_terms_im[6][3] = {{0, 2, 0}, {0, 3, 0}, {1, 2, 0}, {2, 0, 1}, {2, 1, 1}, {3, 0, 1}};

// D_re = Cr Br - Ci Bi, D_im = Cr Bi + Ci Br; conj(C): the Ci terms flip sign.
// The small cross terms (hi*lo, lo*hi) are accumulated first, while the FP32
// accumulator is still small, and the hi*hi terms last: each accumulator
// update rounds at the accumulator's magnitude, so this keeps the number of
// full-magnitude updates per output at 2 * M / 16 instead of 6 * M / 16.
template <bool F16>
__device__ __forceinline__ void issue_sandwich_stage(uint32_t tm, uint32_t bpl_saddr, bool conj) {
  for (int part = 0; part < 2; ++part) {
    const uint32_t d = tm + kColD + 128 * part;
    uint32_t acc = 0;
    for (int phase = 0; phase < 2; ++phase) {
      for (int kk = 0; kk < TM / 16; ++kk) {
        for (int j = 0; j < 6; ++j) {
          const bool main_term = j == 0 || j == 3;  // hi * hi
          if (main_term != (phase == 1)) continue;
          const int* term = part == 0 ? c_terms_re[j] : c_terms_im[j];
          bool neg = false;
          if (term[2]) neg = part == 0 ? !conj : conj;
          const uint32_t a = tm + kColA + 64 * term[0] + 8 * kk;
          const uint64_t b = tc::smem_desc(bpl_saddr + term[1] * kPlaneBytes + kk * 256, 128, 2048);
          tc::mma_ts(d, a, b, tc::idesc_bf16(128, 128, neg, F16), acc);
          acc = 1;
        }
      }
    }
  }
}

}  // namespace

template <int MODE, bool F16>
__global__ void __launch_bounds__(kTcThreads, 1) k_chain_tc(const ChainArgs a, const uint32_t* __restrict__ cplanes) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* bpl = smem;  // 4 planes of the B operand, K-major core-matrix layout
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 4 * kPlaneBytes);
  uint32_t* tbase = reinterpret_cast<uint32_t*>(smem + 4 * kPlaneBytes + 8);
  double* red = reinterpret_cast<double*>(smem + 4 * kPlaneBytes + 16);  // [kTcThreads / 32]
  int* range_flag = reinterpret_cast<int*>(smem + 4 * kPlaneBytes + 16 + 8 * (kTcThreads / 32));
  const int t = threadIdx.x, w = t >> 5;
  const int m = t & 127;    // accumulator row (tensor-memory lane) of this thread
  const int grp = t >> 7;           // column group of this thread
  const int c0 = kTcChunks * grp;   // its 16-column chunks: c0 .. c0 + kTcChunks - 1
  const int il = blockIdx.x, gi = a.pos_begin + il;
  const int2 r = a.pos[gi];
  const int yi = r.x, xi = r.y;
  if (yi < 0 || xi < 0 || yi > a.H - TM || xi > a.W - TM) {
    if (t == 0) {
      *a.status = PTYCHO_ERR_POSITION;
      if (MODE != MODE_FORWARD) a.loss_part[il] = 0.0;
    }
    if (MODE == MODE_GRAD)
      for (int k = t; k < TM * TM; k += blockDim.x) a.ws_gp[(size_t)il * TM * TM + k] = make_float2(0.f, 0.f);
    return;
  }
  if (w == 0) {
    tc::tmem_alloc(tbase, 512);
    tc::tmem_relinquish();
  }
  if (t == 0) {
    tc::mbar_init(mbar, 1);
    *range_flag = 0;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = *tbase;
  const uint32_t trow = tm + ((uint32_t)(32 * (w & 3)) << 16);  // this warp's lane quarter
  const uint32_t bpl_saddr = tc::smem_u32(bpl);
  uint32_t parity = 0;
  const size_t MM = (size_t)TM * TM;
  const size_t HW = (size_t)a.H * a.W;
  const float2* objw = a.obj + (size_t)yi * a.W + xi;
  const float2* dirw = (MODE != MODE_GRAD && a.obj_dir) ? a.obj_dir + (size_t)yi * a.W + xi : nullptr;

  // C planes (0 = propagator K, 1 = DFT F) into tensor-memory columns 256..511.
  auto load_planes = [&](int which) {
    const uint32_t* src = cplanes + (size_t)which * 4 * TM * 64;
    for (int q = (4 / kTcGroups) * grp; q < (4 / kTcGroups) * (grp + 1); ++q)
      for (int c = 0; c < 64; c += 16) {
        uint32_t rr[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) rr[j] = __ldg(src + (size_t)(q * TM + m) * 64 + c + j);
        tc::tmem_st16(trow + kColA + 64 * q + c, rr);
      }
    tc::tmem_wait_st();
  };
  // Row n = m, elements k in [16 c, 16 c + 16) of the B operand planes.
  auto write_b = [&](int c, const float (&re)[16], const float (&im)[16]) {
    uint32_t p[4][8];
    if constexpr (F16) {
      float mx = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) mx = fmaxf(mx, fmaxf(fabsf(re[j]), fabsf(im[j])));
      if (!(mx < 60000.f)) *range_flag = 1;  // outside the half-precision range (or NaN)
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float h0, l0, h1, l1;
      if constexpr (F16) {
        tc::split_f16(re[2 * j], h0, l0);
        tc::split_f16(re[2 * j + 1], h1, l1);
        p[0][j] = tc::pack_f16x2(h0, h1);
        p[1][j] = tc::pack_f16x2(l0, l1);
        tc::split_f16(im[2 * j], h0, l0);
        tc::split_f16(im[2 * j + 1], h1, l1);
        p[2][j] = tc::pack_f16x2(h0, h1);
        p[3][j] = tc::pack_f16x2(l0, l1);
      } else {
        tc::split_bf16(re[2 * j], h0, l0);
        tc::split_bf16(re[2 * j + 1], h1, l1);
        p[0][j] = tc::pack_bf16x2(h0, h1);
        p[1][j] = tc::pack_bf16x2(l0, l1);
        tc::split_bf16(im[2 * j], h0, l0);
        tc::split_bf16(im[2 * j + 1], h1, l1);
        p[2][j] = tc::pack_bf16x2(h0, h1);
        p[3][j] = tc::pack_bf16x2(l0, l1);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kc = 2 * c + h;
        unsigned char* dst = bpl + q * kPlaneBytes + (m % 8) * 16 + kc * 128 + (m / 8) * 2048;
        *reinterpret_cast<uint4*>(dst) = make_uint4(p[q][4 * h], p[q][4 * h + 1], p[q][4 * h + 2], p[q][4 * h + 3]);
      }
  };
  auto read_d = [&](int c, float (&re)[16], float (&im)[16]) {
    uint32_t rr[16], ri[16];
    tc::tmem_ld16(trow + kColD + 16 * c, rr);
    tc::tmem_ld16(trow + kColD + 128 + 16 * c, ri);
    tc::tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      re[j] = __uint_as_float(rr[j]);
      im[j] = __uint_as_float(ri[j]);
    }
  };
  // Issue one MMA stage on the B planes just written and wait for it; false
  // (for every thread) if the tensor core did not finish in time.
  auto stage = [&](bool conj) -> bool {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (t == 0 && !a.selftest_timeout) {
      tc::fence_after_sync();
      issue_sandwich_stage<F16>(tm, bpl_saddr, conj);
      tc::mma_commit(mbar);
    }
    const bool done = tc::mbar_wait_bounded(mbar, parity, kWaitCycles);
    parity ^= 1u;
    tc::fence_after_sync();
    return __syncthreads_and(done) != 0;
  };
  // stage 1, transpose through the B operand, stage 2: D <- (C W C)^T
  auto sandwich = [&](bool conj) -> bool {
    if (!stage(conj)) return false;
    for (int c = c0; c < c0 + kTcChunks; ++c) {
      float re[16], im[16];
      read_d(c, re, im);
      write_b(c, re, im);
    }
    return stage(conj);
  };

  bool ok = true;
  load_planes(0);
  // phi_0 = P * O_0, column-held: thread t owns x = t, rows y = 16 c + j
  for (int c = c0; c < c0 + kTcChunks; ++c) {
    float re[16], im[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int y = 16 * c + j;
      float2 p = __ldg(a.probe + y * TM + m);
      if (a.probe_dir) {
        const float2 d = __ldg(a.probe_dir + y * TM + m);
        p.x = fmaf(a.probe_step, d.x, p.x);
        p.y = fmaf(a.probe_step, d.y, p.y);
      }
      float2 o = __ldg(objw + (size_t)y * a.W + m);
      if (dirw) {
        const float2 d = __ldg(dirw + (size_t)y * a.W + m);
        o.x = fmaf(a.obj_step, d.x, o.x);
        o.y = fmaf(a.obj_step, d.y, o.y);
      }
      const float2 ph = cmul_tc(p, o);
      re[j] = ph.x;
      im[j] = ph.y;
    }
    write_b(c, re, im);
  }
  for (int s = 0; ok && s + 1 < a.S; ++s) {
    ok = sandwich(false);  // D = psi_{s+1}
    if (!ok) break;
    const float2* ow = objw + (size_t)(s + 1) * HW;
    const float2* dw = dirw ? dirw + (size_t)(s + 1) * HW : nullptr;
    float2* wdst = MODE == MODE_GRAD ? a.ws_psi + ((size_t)s * a.ws_n + il) * MM : nullptr;
    for (int c = c0; c < c0 + kTcChunks; ++c) {
      float re[16], im[16];
      read_d(c, re, im);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int y = 16 * c + j;
        if (MODE == MODE_GRAD) __stcs(wdst + y * TM + m, make_float2(re[j], im[j]));
        float2 o = __ldg(ow + (size_t)y * a.W + m);
        if (dw) {
          const float2 d = __ldg(dw + (size_t)y * a.W + m);
          o.x = fmaf(a.obj_step, d.x, o.x);
          o.y = fmaf(a.obj_step, d.y, o.y);
        }
        const float2 ph = cmul_tc(make_float2(re[j], im[j]), o);
        re[j] = ph.x;
        im[j] = ph.y;
      }
      write_b(c, re, im);
    }
  }
  if (ok) {
    tc::fence_before_sync();
    __syncthreads();
    load_planes(1);
    ok = sandwich(false);  // D = far field Psi, column-held (thread t owns kx = t)
  }
  if (ok) {
    if constexpr (MODE == MODE_FORWARD) {
      float2* po = a.psi_out ? a.psi_out + (size_t)gi * MM : nullptr;
      float* io = a.int_out ? a.int_out + (size_t)gi * MM : nullptr;
      for (int c = c0; c < c0 + kTcChunks; ++c) {
        float re[16], im[16];
        read_d(c, re, im);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int ky = 16 * c + j;
          if (po) po[ky * TM + m] = make_float2(re[j], im[j]);
          if (io) io[ky * TM + m] = fmaf(re[j], re[j], im[j] * im[j]);
        }
      }
    } else {
      // Amplitude residual of Eq. 1 and the seed of the adjoint.
      const float* Ii = a.meas + (size_t)gi * MM;
      double lsum = 0.0;
      for (int c = c0; c < c0 + kTcChunks; ++c) {
        float re[16], im[16];
        read_d(c, re, im);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int ky = 16 * c + j;
          const float A = sqrtf(__ldg(Ii + ky * TM + m));
          const float mag = sqrtf(fmaf(re[j], re[j], im[j] * im[j]));
          const float d = mag - A;
          lsum += (double)d * (double)d;
          const float sc = mag > 0.0f ? (2.0f * d) / mag : 0.0f;
          re[j] *= sc;
          im[j] *= sc;
        }
        if (MODE == MODE_GRAD) write_b(c, re, im);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
      if ((t & 31) == 0) red[w] = lsum;
      __syncthreads();
      if (t == 0) {
        double tot = 0.0;
        for (int k = 0; k < kTcThreads / 32; ++k) tot += red[k];
        a.loss_part[il] = tot;
      }
      if constexpr (MODE == MODE_GRAD) {
        ok = sandwich(true);  // g_phi_{S-1} = conj(F) g_Psi conj(F)
        if (ok) {
          tc::fence_before_sync();
          __syncthreads();
          load_planes(0);
        }
        for (int s = a.S - 1; ok && s >= 0; --s) {
          float2* gdst = a.ws_gphi + ((size_t)s * a.ws_n + il) * MM;
          const float2* ow = objw + (size_t)s * HW;
          float2* gp = a.ws_gp + (size_t)il * MM;
          for (int c = c0; c < c0 + kTcChunks; ++c) {
            float re[16], im[16];
            read_d(c, re, im);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int y = 16 * c + j;
              __stcs(gdst + y * TM + m, make_float2(re[j], im[j]));
              const float2 g = cmulc_tc(make_float2(re[j], im[j]), __ldg(ow + (size_t)y * a.W + m));
              re[j] = g.x;
              im[j] = g.y;
              if (s == 0) __stcs(gp + y * TM + m, g);
            }
            if (s > 0) write_b(c, re, im);
          }
          if (s > 0) ok = sandwich(true);
        }
      }
    }
  }
  if (!ok) {
    // The tensor core did not signal completion in time: flag the call, give
    // the outstanding work one more bounded wait, then release tensor memory.
    if (t == 0) {
      *a.status = PTYCHO_ERR_TIMEOUT;
      if (MODE != MODE_FORWARD) a.loss_part[il] = 0.0;
    }
    tc::mbar_wait_bounded(mbar, parity ^ 1u, kWaitCycles);  // the phase that timed out
  }
  tc::fence_before_sync();
  __syncthreads();
  if (F16 && t == 0 && *range_flag) *a.status = PTYCHO_ERR_UNSUPPORTED;
  if (w == 0) tc::tmem_dealloc(tm, 512);
}

size_t chain_tc_smem_bytes() { return 4 * (size_t)kPlaneBytes + 256; }

template <bool F16>
static cudaError_t prepare_tc() {
  const int bytes = (int)chain_tc_smem_bytes();
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_chain_tc<MODE_FORWARD, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_chain_tc<MODE_LOSS, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) !=
      cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_chain_tc<MODE_GRAD, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t chain_tc_prepare() {
  cudaError_t e = prepare_tc<false>();
  return e != cudaSuccess ? e : prepare_tc<true>();
}

template <bool F16>
static cudaError_t launch_tc(ChainMode mode, const ChainArgs& a, const uint32_t* cplanes, cudaStream_t st) {
  const size_t smem = chain_tc_smem_bytes();
  switch (mode) {
    case MODE_FORWARD: k_chain_tc<MODE_FORWARD, F16><<<a.n_pos, kTcThreads, smem, st>>>(a, cplanes); break;
    case MODE_LOSS: k_chain_tc<MODE_LOSS, F16><<<a.n_pos, kTcThreads, smem, st>>>(a, cplanes); break;
    case MODE_GRAD: k_chain_tc<MODE_GRAD, F16><<<a.n_pos, kTcThreads, smem, st>>>(a, cplanes); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_chain_tc(ChainMode mode, const ChainArgs& a, const uint32_t* cplanes, bool f16,
                            cudaStream_t st) {
  if (a.n_pos <= 0) return cudaSuccess;
  return f16 ? launch_tc<true>(mode, a, cplanes, st) : launch_tc<false>(mode, a, cplanes, st);
}

}  // namespace ptycho
