// Generic-window slice chain: any probe window M = 2^a 3^b (8 <= M <= 4096)
// that the register-resident kernels do not cover (they take M = 64, 128).
//
// The chunk's positions advance through the multislice model (Sec. II-B)
// together, slice by slice: their waves live in a global buffer wv[n][M][M].
// Every pass transforms a block of rows or columns of one wave with
// mixed-radix (8/4/2/3) Stockham stages in natural order: the first stage
// reads the lines from the wave, later stages go through shared memory, the
// last writes the lines back.  Because the Fresnel factor is separable, a
// propagation is a row pass and a column pass, each running FFT, factor and
// inverse on its lines; the transmission of a slice and its adjoint ride on
// the row passes.  The amplitude residual of Eq. 1 is one pointwise kernel.
// The workspace it fills (entering waves, exit-wave gradients, probe-gradient
// parts, loss parts) has the layout of the register-resident kernels, so the
// tiled reductions are shared.
#include "../../include/ptycho.h"
#include "fft2d.cuh"
#include "internal.h"

// Line-pass block shape: threads, the most elements (lines x M) a block
// takes, and the resident blocks per SM it is compiled for (register cap).
#ifndef PTYCHO_GM_THREADS
#define PTYCHO_GM_THREADS 256
#endif
#ifndef PTYCHO_GM_ELEMS
#define PTYCHO_GM_ELEMS 4096
#endif
#ifndef PTYCHO_GM_MIN_BLOCKS
#define PTYCHO_GM_MIN_BLOCKS 4
#endif

namespace ptycho {

// Constants of the composite radices (outside the anonymous namespace: not
// every radix is instantiated in every build).
namespace gmr {

// w_R^e = exp(-2 pi i e / R) for the composite radices (the inverse uses the
// conjugate), as exact constants.
template <int R>
struct Wr;
template <>
struct Wr<16> {
  static constexpr float c[16] = {1.f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                                  0.f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                                  -1.f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                                  0.f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
  static constexpr float s[16] = {0.f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                                  -1.f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                                  0.f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                                  1.f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f};
};
template <>
struct Wr<12> {
  static constexpr float c[12] = {1.f, 0.86602540378443865f, 0.5f, 0.f, -0.5f, -0.86602540378443865f,
                                  -1.f, -0.86602540378443865f, -0.5f, 0.f, 0.5f, 0.86602540378443865f};
  static constexpr float s[12] = {0.f, -0.5f, -0.86602540378443865f, -1.f, -0.86602540378443865f, -0.5f,
                                  0.f, 0.5f, 0.86602540378443865f, 1.f, 0.86602540378443865f, 0.5f};
};
template <>
struct Wr<6> {
  static constexpr float c[6] = {1.f, 0.5f, -0.5f, -1.f, -0.5f, 0.5f};
  static constexpr float s[6] = {0.f, -0.86602540378443865f, -0.86602540378443865f, 0.f,
                                 0.86602540378443865f, 0.86602540378443865f};
};

// R = R1 R2 for the composite radices.
template <int R>
struct Split;
template <>
struct Split<16> {
  static constexpr int R1 = 4, R2 = 4;
};
template <>
struct Split<12> {
  static constexpr int R1 = 4, R2 = 3;
};
template <>
struct Split<6> {
  static constexpr int R1 = 2, R2 = 3;
};

}  // namespace gmr

namespace {

// Small DFT of a register array in natural order, forward kernel
// exp(-2 pi i n k / R), inverse its conjugate, unnormalised.
// v w_R^e (forward) or v conj(w_R^e) (inverse), with the trivial factors
// (1, -i, -1, +i) as sign and swap operations.
template <int R, int E, bool INV>
__device__ __forceinline__ float2 mul_wr(float2 v) {
  constexpr int e = E % R;
  if constexpr (e == 0) {
    return v;
  } else if constexpr (4 * e == R) {
    return mul_mi<INV>(v);
  } else if constexpr (2 * e == R) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (4 * e == 3 * R) {
    return mul_mi<!INV>(v);
  } else {
    const float c = gmr::Wr<R>::c[e], sn = INV ? -gmr::Wr<R>::s[e] : gmr::Wr<R>::s[e];
    return make_float2(fmaf(v.x, c, -v.y * sn), fmaf(v.x, sn, v.y * c));
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2 (&x)[R]);

// Composite small DFT (one Cooley-Tukey step in registers): with n = R2 n1 + n2
// and k = k1 + R1 k2, X[k] = sum_n2 w_R2^(n2 k2) w_R^(n2 k1) sum_n1 w_R1^(n1 k1) x[n].
template <int R, bool INV>
__device__ __forceinline__ void dft_composite(float2 (&x)[R]) {
  constexpr int R1 = gmr::Split<R>::R1, R2 = gmr::Split<R>::R2;
  float2 y[R];  // y[n2 R1 + k1]
  static_for<0, R2>([&](auto n2c) {
    constexpr int n2 = decltype(n2c)::value;
    float2 u[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) u[n1] = x[R2 * n1 + n2];
    dft_r<R1, INV>(u);
    static_for<0, R1>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      y[n2 * R1 + k1] = mul_wr<R, n2 * k1, INV>(u[k1]);
    });
  });
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    float2 u[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) u[n2] = y[n2 * R1 + k1];
    dft_r<R2, INV>(u);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = u[k2];
  }
}

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
  } else if constexpr (R == 8) {
    dft8<INV>(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7]);
  } else {
    static_assert(R == 6 || R == 12 || R == 16, "radix 2, 3, 4, 6, 8, 12 or 16");
    dft_composite<R, INV>(x);
  }
}

// Shared-memory slot of element i of a line: one padding slot every 16
// elements, which spreads the radix-8 first stage (outputs 8 apart across
// threads) over the banks; the odd line stride does the same for the column
// transposes.  (Simulated bank wavefronts per warp access, ideal 2: 2.0-2.8
// for M = 96, 192, 256 against 3.3-4.7 unpadded.)
__host__ __device__ constexpr int gm_pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int gm_line_stride(int M) { return M + M / 16 + 1; }

// Radix schedule of a window: with big, greedily the largest radix of 16, 12,
// 8, 6, 4, 3, 2 that divides what is left (fewer stages: fewer shared-memory
// round trips, more registers per thread); else 8s, then 4, 2, 3.  Which
// instances take the large radices is in GmTraits.
#ifndef PTYCHO_GM_MAX_RADIX
#define PTYCHO_GM_MAX_RADIX 16
#endif
__host__ __device__ constexpr int gm_radix_at(int M, int i, bool big = false) {
  int m = M, k = 0;
  const int order16[7] = {16, 12, 8, 6, 4, 3, 2};
  const int order8[4] = {8, 4, 2, 3};
  const bool b = big && PTYCHO_GM_MAX_RADIX >= 16;
  const int* order = b ? order16 : order8;
  const int n_order = b ? 7 : 4;
  for (int o = 0; o < n_order; ++o)
    while (m % order[o] == 0 && m > 1) {
      if (k == i) return order[o];
      m /= order[o];
      ++k;
    }
  return 0;
}
__host__ __device__ constexpr int gm_n_stages(int M, bool big = false) {
  int n = 0;
  while (gm_radix_at(M, n, big) != 0) ++n;
  return n;
}
constexpr int kGmThreads = PTYCHO_GM_THREADS;

// Per-instance choices, measured on the batched workload's windows (chain
// time of all its problems of that window): the large radices (16/12/6) and a
// 128-register budget (2 blocks/SM) win for 256 (197 vs 215 ms); 96 takes the
// large radices at 80 registers (39 vs 42 ms); 192 keeps radix 8 at 64
// registers and 256 threads (368 ms against 385-405 ms with radix 12/16,
// and 378-402 ms with 192, 384 or 512 threads per block; 16 lines per block
// against 32 or 64: 406 against 468 and 581 ms for the 192 problems alone).
// The paper's 1024 window takes radices 16 16 4 at 128 registers and 4 lines
// per block (143 positions/s at 100 slices, against 117 with radix 8 at 64
// registers, 131 and 140 with 2 and 8 lines per block).
#ifndef PTYCHO_GM192_THREADS
#define PTYCHO_GM192_THREADS 256
#endif
#ifndef PTYCHO_GM192_MIN_BLOCKS
#define PTYCHO_GM192_MIN_BLOCKS PTYCHO_GM_MIN_BLOCKS
#endif
template <int MC>
struct GmTraits {
  static constexpr bool big = false;
  static constexpr int min_blocks = PTYCHO_GM_MIN_BLOCKS;
  static constexpr int threads = kGmThreads;
};
template <>
struct GmTraits<256> {
  static constexpr bool big = PTYCHO_GM_MAX_RADIX >= 16;
  static constexpr int min_blocks = 2;
  static constexpr int threads = kGmThreads;
};
template <>
struct GmTraits<96> {
  static constexpr bool big = PTYCHO_GM_MAX_RADIX >= 16;
  static constexpr int min_blocks = 3;
  static constexpr int threads = kGmThreads;
};
#ifndef PTYCHO_GM1024_BIG
#define PTYCHO_GM1024_BIG 1
#endif
#ifndef PTYCHO_GM1024_MIN_BLOCKS
#define PTYCHO_GM1024_MIN_BLOCKS 2
#endif
template <>
struct GmTraits<1024> {  // the paper's detector size (Table I): radices 16 16 4
  static constexpr bool big = PTYCHO_GM_MAX_RADIX >= 16 && PTYCHO_GM1024_BIG;
  static constexpr int min_blocks = PTYCHO_GM1024_MIN_BLOCKS;
  static constexpr int threads = kGmThreads;
};
template <>
struct GmTraits<192> {
  static constexpr bool big = false;
  static constexpr int min_blocks = PTYCHO_GM192_MIN_BLOCKS;
  static constexpr int threads = PTYCHO_GM192_THREADS;
};

// Lines per block: the largest divisor of M with L M <= PTYCHO_GM_ELEMS.
#ifndef PTYCHO_GM192_LINES
#define PTYCHO_GM192_LINES 0
#endif
#ifndef PTYCHO_GM1024_LINES
#define PTYCHO_GM1024_LINES 0
#endif
__host__ __device__ constexpr int gm_lines(int M) {
  if (M == 192 && PTYCHO_GM192_LINES > 0) return PTYCHO_GM192_LINES;
  if (M == 1024 && PTYCHO_GM1024_LINES > 0) return PTYCHO_GM1024_LINES;
  int best = 1;
  for (int L = 1; L <= M && L * M <= PTYCHO_GM_ELEMS; ++L)
    if (M % L == 0) best = L;
  return best;
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

// Where a stage takes its inputs and puts its outputs: the block's shared
// line buffers, the same times the propagation factor, or the wave in global
// memory (first and last stage of a transform).
enum : int { IO_SMEM = 0, IO_SMEM_H = 1, IO_GLOBAL = 2 };

// The block's lines and what its first and last stages do with global
// memory.  MC > 0: the window is a compile-time constant.
template <int MC>
struct GmCtx {
  const ChainArgs& a;
  GmLineArgs g;
  int m, l;              // window and lines per block (when MC == 0)
  int l0, il;            // first line, position in the chunk
  int2 r;                // window corner (y, x)
  bool ok, from_probe;
  float2* base;          // this position's wave
  const float2* in;      // row source of the first stage: the wave, or the probe at s = 0
  const float2* Tst;     // per-stage twiddles (shared)
  const float2* Hs;      // propagation factor hs[k] (shared)

  __device__ __forceinline__ int M() const {
    if constexpr (MC > 0) return MC; else return m;
  }
  __device__ __forceinline__ int L() const {
    if constexpr (MC > 0) return gm_lines(MC); else return l;
  }
  // (y, x) and offset in the wave of element i of line li
  __device__ __forceinline__ int y_of(int li, int i) const { return g.cols ? i : l0 + li; }
  __device__ __forceinline__ int x_of(int li, int i) const { return g.cols ? l0 + li : i; }
  __device__ __forceinline__ size_t at(int li, int i) const { return (size_t)y_of(li, i) * M() + x_of(li, i); }
  __device__ __forceinline__ size_t obj_at(int li, int i) const {
    return (size_t)g.s * a.H * a.W + (size_t)(r.x + y_of(li, i)) * a.W + (r.y + x_of(li, i));
  }

  // x[q] = element i0 + q di of line li, with the forward transmission when
  // the pass carries it: all loads are issued before any is used.
  template <int R>
  __device__ __forceinline__ void load(float2 (&x)[R], int li, int i0, int di) const {
    const size_t MM = (size_t)M() * M();
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = in[at(li, i0 + q * di)];
    if (!g.pre) return;
    if (!ok) {
#pragma unroll
      for (int q = 0; q < R; ++q) x[q] = make_float2(0.f, 0.f);
      return;
    }
    float2 o[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const size_t oi = obj_at(li, i0 + q * di);
      o[q] = a.obj[oi];
      if (a.obj_dir) {
        const float2 d = a.obj_dir[oi];
        o[q].x = fmaf(a.obj_step, d.x, o[q].x);
        o[q].y = fmaf(a.obj_step, d.y, o[q].y);
      }
      if (from_probe && a.probe_dir) {
        const float2 d = a.probe_dir[at(li, i0 + q * di)];
        x[q].x = fmaf(a.probe_step, d.x, x[q].x);
        x[q].y = fmaf(a.probe_step, d.y, x[q].y);
      }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (g.store) __stcs(a.ws_psi + ((size_t)(g.s - 1) * a.ws_n + il) * MM + at(li, i0 + q * di), x[q]);
      x[q] = cmul(x[q], o[q]);
    }
  }

  // element i0 + q di of line li = x[q], with the adjoint transmission when
  // the pass carries it.
  template <int R>
  __device__ __forceinline__ void store(const float2 (&x)[R], int li, int i0, int di) const {
    const size_t MM = (size_t)M() * M();
    if (!g.post) {
#pragma unroll
      for (int q = 0; q < R; ++q) base[at(li, i0 + q * di)] = x[q];
      return;
    }
    if (!ok) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const size_t e = at(li, i0 + q * di);
        base[e] = make_float2(0.f, 0.f);
        if (g.s == 0) __stcs(a.ws_gp + (size_t)il * MM + e, make_float2(0.f, 0.f));
      }
      return;
    }
    float2 o[R];
#pragma unroll
    for (int q = 0; q < R; ++q) o[q] = a.obj[obj_at(li, i0 + q * di)];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const size_t e = at(li, i0 + q * di);
      __stcs(a.ws_gphi + ((size_t)g.s * a.ws_n + il) * MM + e, x[q]);
      const float2 gv = cmulc(x[q], o[q]);
      if (g.s == 0)
        __stcs(a.ws_gp + (size_t)il * MM + e, gv);
      else
        base[e] = gv;
    }
  }
};

// One Stockham autosort stage of radix R over the block's L lines of length
// M, after spans of Ns: butterfly j takes x[j + q M/R], twiddles it by
// w_{Ns R}^{q (j mod Ns)} (per-stage table at toff, contiguous in j mod Ns),
// and writes y[(j - k) R + k + q Ns].  Rows map consecutive threads to
// consecutive butterflies of a line, columns to the same butterfly of
// consecutive lines, so the global first and last stages read and write
// contiguous addresses; in the last stage (Ns = M/R) outputs land at j + q Ns
// in natural order, so the propagation factor can be applied there.
template <int R, bool INV, int IN, int OUT, int MC>
__device__ __forceinline__ void gm_stage(const GmCtx<MC>& c, const float2* __restrict__ src,
                                         float2* __restrict__ dst, int Ns, int toff, bool cj, int t) {
  const int M = c.M(), L = c.L(), LS = gm_line_stride(M);
  const int nb = M / R;
  for (int idx = t; idx < L * nb; idx += GmTraits<MC>::threads) {
    int li, j;
    if (c.g.cols) {
      j = idx / L;
      li = idx - j * L;
    } else {
      li = idx / nb;
      j = idx - li * nb;
    }
    const int k = j % Ns;
    float2 x[R];
    if constexpr (IN == IO_GLOBAL) {
      c.template load<R>(x, li, j, nb);
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) x[q] = src[li * LS + gm_pad(j + q * nb)];
    }
    if (Ns > 1) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        const float2 w = c.Tst[toff + (q - 1) * Ns + k];
        x[q] = INV ? cmulc(x[q], w) : cmul(x[q], w);
      }
    }
    dft_r<R, INV>(x);
    const int d0 = (j - k) * R + k;
    if constexpr (OUT == IO_GLOBAL) {
      c.template store<R>(x, li, d0, Ns);
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int i = d0 + q * Ns;
        float2 v = x[q];
        if constexpr (OUT == IO_SMEM_H) v = cj ? cmulc(v, c.Hs[i]) : cmul(v, c.Hs[i]);
        dst[li * LS + gm_pad(i)] = v;
      }
    }
  }
}

// All stages of one transform of the block's lines, with the schedule known
// at compile time.  Stage i reads the previous stage's buffer (stage 0: `rd`
// or global memory) and writes b0 (i even) or b1 (i odd); returns the buffer
// the last stage wrote when it writes shared memory.
template <bool INV, int IN, int OUT, int MC, int I = 0, int NS = 1, int TOFF = 0>
__device__ __forceinline__ float2* gm_tf_ct(const GmCtx<MC>& c, const float2* rd, float2* b0, float2* b1, bool cj,
                                            int t) {
  constexpr int NST = gm_n_stages(MC, GmTraits<MC>::big);
  constexpr int R = gm_radix_at(MC, I, GmTraits<MC>::big);
  constexpr bool LAST = I == NST - 1;
  float2* wr = (I % 2 == 0) ? b0 : b1;
  gm_stage<R, INV, I == 0 ? IN : IO_SMEM, LAST ? OUT : IO_SMEM, MC>(c, rd, wr, NS, TOFF, cj, t);
  if constexpr (LAST) {
    return wr;
  } else {
    __syncthreads();
    return gm_tf_ct<INV, IN, OUT, MC, I + 1, NS * R, TOFF + (NS > 1 ? (R - 1) * NS : 0)>(c, wr, b0, b1, cj, t);
  }
}

// The same with the schedule read from the plan.
template <int R, bool INV, int IN, int OUT>
__device__ __forceinline__ void gm_stage_rt(const GmCtx<0>& c, const float2* rd, float2* wr, int Ns, int toff,
                                            bool cj, bool first, bool last, int t) {
  if (first && last)
    gm_stage<R, INV, IN, OUT, 0>(c, rd, wr, Ns, toff, cj, t);
  else if (first)
    gm_stage<R, INV, IN, IO_SMEM, 0>(c, rd, wr, Ns, toff, cj, t);
  else if (last)
    gm_stage<R, INV, IO_SMEM, OUT, 0>(c, rd, wr, Ns, toff, cj, t);
  else
    gm_stage<R, INV, IO_SMEM, IO_SMEM, 0>(c, rd, wr, Ns, toff, cj, t);
}

template <bool INV, int IN, int OUT>
__device__ __forceinline__ float2* gm_tf_rt(const GmCtx<0>& c, const GmPlan& plan, const float2* rd, float2* b0,
                                            float2* b1, bool cj, int t) {
  int Ns = 1, toff = 0;
  float2* wr = b0;
  for (int i = 0; i < plan.n; ++i) {
    const int R = plan.r[i];
    const bool first = i == 0, last = i == plan.n - 1;
    wr = (i % 2 == 0) ? b0 : b1;
    if (R == 8)
      gm_stage_rt<8, INV, IN, OUT>(c, rd, wr, Ns, toff, cj, first, last, t);
    else if (R == 4)
      gm_stage_rt<4, INV, IN, OUT>(c, rd, wr, Ns, toff, cj, first, last, t);
    else if (R == 2)
      gm_stage_rt<2, INV, IN, OUT>(c, rd, wr, Ns, toff, cj, first, last, t);
    else
      gm_stage_rt<3, INV, IN, OUT>(c, rd, wr, Ns, toff, cj, first, last, t);
    if (!last) __syncthreads();
    if (Ns > 1) toff += (R - 1) * Ns;
    Ns *= R;
    rd = wr;
  }
  return wr;
}

template <bool INV, int IN, int OUT, int MC>
__device__ __forceinline__ float2* gm_tf(const GmCtx<MC>& c, const GmPlan& plan, const float2* rd, float2* b0,
                                         float2* b1, bool cj, int t) {
  if constexpr (MC > 0)
    return gm_tf_ct<INV, IN, OUT, MC>(c, rd, b0, b1, cj, t);
  else
    return gm_tf_rt<INV, IN, OUT>(c, plan, rd, b0, b1, cj, t);
}

// One pass over L rows or columns of each wave.  The Fresnel factor is
// separable, h(ky, kx) = h1(ky) h1(kx), so a propagation F^-1 h F is a 1-D
// propagation of every row followed by one of every column: each pass runs
// FFT, the factor hs[k] = h1(k)/M (applied by the FFT's last stage) and the
// inverse on its lines, reading them from the wave in its first stage and
// writing them back in its last.  Row passes also apply the slice's
// transmission (Sec. II-B) on load, or its adjoint on store, so a slice
// costs one row and one column pass each way.
//   forward transmission (pre):  psi_0 = P (+ step dir); [psi_s -> workspace];
//                                v = psi_s O_s[window] (+ step dir)
//   adjoint transmission (post): g_phi_s -> workspace, v = conj(O_s[window]) g_phi_s,
//                                at s = 0 into the probe-gradient workspace instead.
// Skipped (out-of-range) windows carry zeros and flag the call.
template <int MC>
__global__ void __launch_bounds__(GmTraits<MC>::threads, GmTraits<MC>::min_blocks) k_gm_line(const ChainArgs a, float2* __restrict__ wv, int M, GmPlan plan,
                                                 GmLineArgs g) {
  if constexpr (MC > 0) M = MC;
  const int L = MC > 0 ? gm_lines(MC) : gm_lines(M);
  const int LS = gm_line_stride(M);
  extern __shared__ float2 gsm[];
  float2* A = gsm;
  float2* B = A + (size_t)L * LS;
  float2* Tst = B + (size_t)L * LS;  // sum over stages of (R - 1) Ns < M entries
  float2* Hs = Tst + M;
  const int t = threadIdx.x;
  {
    const int nst = MC > 0 ? gm_n_stages(MC, GmTraits<MC>::big) : plan.n;
    int Ns = 1, toff = 0;
    for (int i = 0; i < nst; ++i) {
      const int R = MC > 0 ? gm_radix_at(MC, i, GmTraits<MC>::big) : plan.r[i];
      if (Ns > 1) {
        const int tstep = M / (Ns * R);
        for (int e = t; e < (R - 1) * Ns; e += GmTraits<MC>::threads) {
          const int q = 1 + e / Ns, k = e - (q - 1) * Ns;
          Tst[toff + e] = a.tw[tstep * q * k];
        }
        toff += (R - 1) * Ns;
      }
      Ns *= R;
    }
    for (int k = t; k < M; k += GmTraits<MC>::threads) Hs[k] = a.hs[k];
  }
  const int g0 = blockIdx.x * L;  // first line of this block (L divides M)
  const int il = g0 / M;
  const int l0 = g0 - il * M;
  float2* base = wv + (size_t)il * M * M;
  const int2 r = a.pos[a.pos_begin + il];
  const bool ok = window_ok(r, M, a.H, a.W);
  const bool from_probe = g.pre && g.s == 0;
  const GmCtx<MC> c{a, g, M, L, l0, il, r, ok, from_probe, base, from_probe ? a.probe : base, Tst, Hs};
  if (g.pre && !ok && l0 == 0 && t == 0) *a.status = PTYCHO_ERR_POSITION;
  __syncthreads();
  if (g.op == GM_FFT) {
    gm_tf<false, IO_GLOBAL, IO_GLOBAL, MC>(c, plan, nullptr, A, B, false, t);
  } else if (g.op == GM_IFFT) {
    gm_tf<true, IO_GLOBAL, IO_GLOBAL, MC>(c, plan, nullptr, A, B, false, t);
  } else {
    const bool cj = g.op == GM_PROP_CONJ;
    float2* spec = gm_tf<false, IO_GLOBAL, IO_SMEM_H, MC>(c, plan, nullptr, A, B, cj, t);
    __syncthreads();
    gm_tf<true, IO_SMEM, IO_GLOBAL, MC>(c, plan, spec, spec == A ? B : A, spec, cj, t);
  }
}

// Far field (unnormalised: M Psi) -> outputs (forward mode) or the residual
// of Eq. 1: loss part per position (FP64, fixed order) and the adjoint seed
// 2 d Psi/|Psi| / M, pre-scaled for the unnormalised inverse.  One block of
// 1024 threads per position; each thread loads U elements before using them.
template <int MODE>
__global__ void __launch_bounds__(1024) k_gm_residual(const ChainArgs a, float2* __restrict__ wv, int M) {
  constexpr int NT = 1024, U = 4;
  __shared__ double red[NT / 32];
  const int il = blockIdx.x, gi = a.pos_begin + il, t = threadIdx.x;
  const int MM = M * M;
  float2* w = wv + (size_t)il * MM;
  const bool ok = window_ok(a.pos[gi], M, a.H, a.W);
  const float inv_m = 1.0f / (float)M;
  if (MODE == MODE_FORWARD) {
    if (!ok) return;
    for (int k = t; k < MM; k += NT) {
      const float2 z = make_float2(w[k].x * inv_m, w[k].y * inv_m);
      if (a.psi_out) a.psi_out[(size_t)gi * MM + k] = z;
      if (a.int_out) a.int_out[(size_t)gi * MM + k] = fmaf(z.x, z.x, z.y * z.y);
    }
    return;
  }
  double lsum = 0.0;
  const float* Ii = a.meas + (size_t)gi * MM;
  for (int k0 = 0; k0 < MM; k0 += NT * U) {
    float2 z[U];
    float I[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * NT + t;
      if (k < MM && ok) {
        z[u] = w[k];
        I[u] = Ii[k];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * NT + t;
      if (k >= MM) continue;
      if (!ok) {
        w[k] = make_float2(0.f, 0.f);
        continue;
      }
      const float A = sqrtf(I[u]);
      const float mag = sqrtf(fmaf(z[u].x, z[u].x, z[u].y * z[u].y));
      const float d = mag * inv_m - A;
      lsum += (double)d * (double)d;
      const float sc = mag > 0.0f ? (2.0f * d) / (mag * (float)M) : 0.0f;
      w[k] = make_float2(z[u].x * sc, z[u].y * sc);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
  if ((t & 31) == 0) red[t >> 5] = lsum;
  __syncthreads();
  if (t == 0) {
    double tot = 0.0;
    for (int k = 0; k < NT / 32; ++k) tot += red[k];
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
  if ((e = gm_set_smem<1024>((int)gm_fft_smem_bytes(1024))) != cudaSuccess) return e;
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

  // The kernel keeps psi_s in ws_psi slot s - 1 and g_phi_s in ws_gphi slot
  // s; another slot (recompute mode) is reached by shifting the launch's
  // workspace pointers by whole slots, so the kernel's addressing (and its
  // register budget) stays the same.
  cudaError_t line(int op, int cols, int s = 0, int pre = 0, int post = 0, int store = 0, int psi_slot = -1,
                   int gphi_slot = -1) {
    const GmLineArgs g{op, cols, s, pre, post, store};
    ChainArgs la = a;
    const size_t slot_elems = (size_t)a.ws_n * M * M;
    if (store && psi_slot >= 0)
      la.ws_psi = reinterpret_cast<float2*>(reinterpret_cast<uintptr_t>(a.ws_psi) +
                                            (uintptr_t)((int64_t)(psi_slot - (s - 1)) * (int64_t)slot_elems *
                                                        (int64_t)sizeof(float2)));
    if (post && gphi_slot >= 0)
      la.ws_gphi = reinterpret_cast<float2*>(reinterpret_cast<uintptr_t>(a.ws_gphi) +
                                             (uintptr_t)((int64_t)(gphi_slot - s) * (int64_t)slot_elems *
                                                         (int64_t)sizeof(float2)));
    const unsigned grid = (unsigned)((size_t)a.n_pos * M / gm_lines(M));
    const size_t smem = gm_fft_smem_bytes(M);
    switch (M) {
      case 96: k_gm_line<96><<<grid, GmTraits<96>::threads, smem, st>>>(la, wv, M, plan, g); break;
      case 192: k_gm_line<192><<<grid, GmTraits<192>::threads, smem, st>>>(la, wv, M, plan, g); break;
      case 256: k_gm_line<256><<<grid, GmTraits<256>::threads, smem, st>>>(la, wv, M, plan, g); break;
      case 1024: k_gm_line<1024><<<grid, GmTraits<1024>::threads, smem, st>>>(la, wv, M, plan, g); break;
      default: k_gm_line<0><<<grid, kGmThreads, smem, st>>>(la, wv, M, plan, g); break;
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
//
// Recompute mode (ckpt_L = L, K = ceil(S / L) segments) follows the
// register-resident kernels' schedule with the chunk's waves in wv:
// MODE_GRAD_RC runs the forward keeping the waves entering segments 1..K-2
// (ws_psi slots 0..K-3) and the last segment's waves (slots K-2 ..), the
// residual, the adjoint through the last segment (g_phi in ws_gphi slots
// s - s0) and parks wv (slot K-2+L); MODE_RC_SEG rebuilds segment a.seg's
// waves from its checkpoint (or the probe), restores the parked state, runs
// the adjoint through the segment and parks it again.  The caller sums each
// segment's (psi, g_phi) pairs into the object gradient in between.
cudaError_t launch_chain_gm(ChainMode mode, const ChainArgs& a, float2* wv, int M, int* n_launches,
                            cudaStream_t st) {
  if (a.n_pos <= 0) return cudaSuccess;
  GmLauncher g{a, wv, M, GmPlan{}, st};
  if (!gm_supported(M, &g.plan)) return cudaErrorInvalidValue;
  cudaError_t e;
  const size_t MM = (size_t)M * M;
  const int L = a.ckpt_L > 0 ? a.ckpt_L : 1;
  const int K = (a.S + L - 1) / L;
  const int seg_slot = K - 2, park_slot = K - 2 + L;
  // wv <-> workspace slot (this launch's positions)
  auto copy = [&](float2* dst, const float2* src) {
    return cudaMemcpyAsync(dst, src, (size_t)a.n_pos * MM * sizeof(float2), cudaMemcpyDeviceToDevice, st);
  };
  auto slot = [&](int k) { return a.ws_psi + (size_t)k * a.ws_n * MM; };
  // adjoint through slices s_hi .. s_lo, g_phi_s into slot s - gbase
  auto adjoint = [&](int s_hi, int s_lo, int gbase) -> cudaError_t {
    for (int s = s_hi; s >= s_lo; --s) {
      const int op = s == a.S - 1 ? GM_IFFT : GM_PROP_CONJ;
      cudaError_t r;
      if ((r = g.line(op, 1)) != cudaSuccess) return r;
      if ((r = g.line(op, 0, s, 0, 1, 0, 0, s - gbase)) != cudaSuccess) return r;
    }
    return cudaSuccess;
  };
  if (mode == MODE_RC_SEG) {
    const int j = a.seg, s0 = j * L, s1 = s0 + L;
    if (j > 0 && (e = copy(wv, slot(j - 1))) != cudaSuccess) return e;
    for (int s = s0; s < s1 - 1; ++s) {
      if ((e = g.line(GM_PROP, 0, s, 1, 0, s > 0, seg_slot + (s - s0))) != cudaSuccess) return e;
      if ((e = g.line(GM_PROP, 1)) != cudaSuccess) return e;
    }
    if (s1 - 1 > 0 && (e = copy(slot(seg_slot + L - 1), wv)) != cudaSuccess) return e;
    if ((e = copy(wv, slot(park_slot))) != cudaSuccess) return e;
    if ((e = adjoint(s1 - 1, s0, s0)) != cudaSuccess) return e;
    if (j > 0 && (e = copy(slot(park_slot), wv)) != cudaSuccess) return e;
    if (n_launches) *n_launches = g.launches;
    return cudaSuccess;
  }
  const bool grad = mode == MODE_GRAD, rc = mode == MODE_GRAD_RC;
  const int s_last = (K - 1) * L;  // first slice of the last segment (recompute mode)
  for (int s = 0; s < a.S; ++s) {
    const bool last = s == a.S - 1;
    const int op = last ? GM_FFT : GM_PROP;
    int store = 0, ps = 0;
    if (grad && s > 0) {
      store = 1;
      ps = s - 1;
    } else if (rc && s > 0 && s % L == 0 && s / L <= K - 2) {
      store = 1;
      ps = s / L - 1;
    } else if (rc && s >= s_last) {
      store = 1;
      ps = seg_slot + (s - s_last);
    }
    if ((e = g.line(op, 0, s, 1, 0, store, ps)) != cudaSuccess) return e;
    if ((e = g.line(op, 1)) != cudaSuccess) return e;
  }
  switch (mode) {
    case MODE_FORWARD: k_gm_residual<MODE_FORWARD><<<a.n_pos, 1024, 0, st>>>(a, wv, M); break;
    case MODE_LOSS: k_gm_residual<MODE_LOSS><<<a.n_pos, 1024, 0, st>>>(a, wv, M); break;
    default: k_gm_residual<MODE_GRAD><<<a.n_pos, 1024, 0, st>>>(a, wv, M); break;
  }
  ++g.launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (grad && (e = adjoint(a.S - 1, 0, 0)) != cudaSuccess) return e;
  if (rc) {
    if ((e = adjoint(a.S - 1, s_last, s_last)) != cudaSuccess) return e;
    if ((e = copy(slot(park_slot), wv)) != cudaSuccess) return e;
  }
  if (n_launches) *n_launches = g.launches;
  return cudaSuccess;
}

}  // namespace ptycho
