// Register-resident 2-D FFT of one M x M complex64 tile per thread block.
//
// The multislice model (Sec. II-B) Fourier transforms each slice's wave,
// multiplies by the propagator and inverse transforms it; the exit wave is
// transformed once more to the detector.  Here one thread block owns one
// probe position's M x M wave for the whole slice chain: each thread keeps
// V = M*M/T complex values in registers and the transform is three radix
// passes, each a 2-D pass that applies one mixed-radix digit of y and one of
// x at once (decimation in frequency).  Between passes the wave is exchanged
// through shared memory in a swizzled row-major layout that is free of bank
// conflicts for all three access patterns.
//
// Forward passes leave the spectrum in digit-reversed storage order; the
// inverse passes undo the forward ones exactly in reverse order on the same
// storage.  So propagate = fwd, pointwise multiply, inv needs no reordering,
// and the register grouping before pass 1 equals the grouping after inverse
// pass 1: consecutive slices chain without any extra exchange.
//
// Transforms here are unnormalised; callers fold the orthonormal 1/M factors
// into the propagator table or the residual.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>

namespace ptycho {

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
template <bool CONJ>
__device__ __forceinline__ float2 cmul_opt(float2 a, float2 b) { return CONJ ? cmulc(a, b) : cmul(a, b); }

// multiply by -i (forward kernel) or +i (inverse kernel)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Small DFTs in natural order, forward kernel exp(-2 pi i n k / R), inverse
// kernel its conjugate, both unnormalised.
__device__ __forceinline__ void dft2(float2& x0, float2& x1) {
  const float2 t = x0;
  x0 = cadd(t, x1);
  x1 = csub(t, x1);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
  const float2 t2 = cadd(x1, x3), t3 = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2& x0, float2& x1, float2& x2, float2& x3,
                                     float2& x4, float2& x5, float2& x6, float2& x7) {
  dft4<INV>(x0, x2, x4, x6);  // even samples -> E0..E3
  dft4<INV>(x1, x3, x5, x7);  // odd samples  -> O0..O3
  const float r = 0.70710678118654752440f;
  // O_k *= w8^k, w8 = exp(-+ 2 pi i / 8)
  const float2 o1 = INV ? make_float2((x3.x - x3.y) * r, (x3.x + x3.y) * r)
                        : make_float2((x3.x + x3.y) * r, (x3.y - x3.x) * r);
  const float2 o2 = mul_mi<INV>(x5);
  const float2 o3 = INV ? make_float2((-x7.x - x7.y) * r, (x7.x - x7.y) * r)
                        : make_float2((x7.y - x7.x) * r, (-x7.x - x7.y) * r);
  const float2 e0 = x0, e1 = x2, e2 = x4, e3 = x6, o0 = x1;
  x0 = cadd(e0, o0); x4 = csub(e0, o0);
  x1 = cadd(e1, o1); x5 = csub(e1, o1);
  x2 = cadd(e2, o2); x6 = csub(e2, o2);
  x3 = cadd(e3, o3); x7 = csub(e3, o3);
}

template <int R, bool INV, int OFF, int ST, int N>
__device__ __forceinline__ void dft_at(float2 (&v)[N]) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2(v[OFF], v[OFF + ST]);
  } else if constexpr (R == 4) {
    dft4<INV>(v[OFF], v[OFF + ST], v[OFF + 2 * ST], v[OFF + 3 * ST]);
  } else if constexpr (R == 8) {
    dft8<INV>(v[OFF], v[OFF + ST], v[OFF + 2 * ST], v[OFF + 3 * ST],
              v[OFF + 4 * ST], v[OFF + 5 * ST], v[OFF + 6 * ST], v[OFF + 7 * ST]);
  } else {
    static_assert(R == 1 || R == 2 || R == 4 || R == 8, "unsupported radix");
  }
}

// ---------------------------------------------------------------------------
// Tile configurations.  Storage index of y: py = d0*SY0 + d1*SY1 + d2 with
// digit j in [0, RY(j)); likewise px for x.  Pass j transforms digit j of y
// and of x.  base<J>(t, q) returns the storage coordinates of the (a=0, b=0)
// element of the q-th group that thread t owns in pass J; element (a, b) of
// that group sits at (py + a*SY(J), px + b*SX(J)).  swz() permutes columns
// inside each 16-element block of a row (bank-conflict-free exchanges).
// ---------------------------------------------------------------------------
template <int M>
struct Cfg;

template <>
struct Cfg<128> {
  static constexpr int M = 128, T = 512, V = 32, MIN_BLOCKS = 1;
  static constexpr int ry(int j) { return j == 0 ? 8 : 4; }
  static constexpr int rx(int j) { return j == 1 ? 8 : 4; }
  static constexpr int sy(int j) { return j == 0 ? 16 : (j == 1 ? 4 : 1); }
  static constexpr int sx(int j) { return j == 0 ? 32 : (j == 1 ? 4 : 1); }
  __device__ static __forceinline__ int swz(int px) { return px ^ (5 * ((px >> 5) & 3)); }
  // The pass-1 <-> pass-2 exchange stays inside warp pairs {2k, 2k+1}: a
  // 64-thread named barrier (ids 1..8) orders it.
  __device__ static __forceinline__ void sync12(int t) {
    asm volatile("bar.sync %0, 64;" ::"r"(1 + (t >> 6)) : "memory");
  }
  template <int J>
  __device__ static __forceinline__ void base(int t, int q, int& py, int& px) {
    const int w = t >> 5, l = t & 31;
    if constexpr (J == 0) {
      py = w; px = l;
    } else if constexpr (J == 1) {
      const int e3 = l & 3, e1 = (l >> 2) & 3;
      const int d3 = ((l >> 4) & 1) | ((w & 1) << 1), d1 = w >> 1;
      py = 16 * d1 + d3; px = 32 * e1 + e3;
    } else {
      const int e1 = l & 3, e2 = l >> 2, g = 2 * w + q;
      py = 16 * (g >> 2) + 4 * (g & 3); px = 32 * e1 + 4 * e2;
    }
  }
};

template <>
struct Cfg<64> {
  static constexpr int M = 64, T = 128, V = 32, MIN_BLOCKS = 4;
  static constexpr int ry(int) { return 4; }
  static constexpr int rx(int) { return 4; }
  static constexpr int sy(int j) { return j == 0 ? 16 : (j == 1 ? 4 : 1); }
  static constexpr int sx(int j) { return j == 0 ? 16 : (j == 1 ? 4 : 1); }
  __device__ static __forceinline__ int swz(int px) { return px ^ (5 * ((px >> 4) & 3)); }
  // The pass-1 <-> pass-2 exchange stays inside each warp.
  __device__ static __forceinline__ void sync12(int) { __syncwarp(); }
  template <int J>
  __device__ static __forceinline__ void base(int t, int q, int& py, int& px) {
    const int w = t >> 5, l = t & 31;
    if constexpr (J == 0) {
      py = (l >> 4) | (w << 1) | (q << 3); px = l & 15;
    } else if constexpr (J == 1) {
      const int e3 = l & 3, e1 = (l >> 2) & 3, d3 = ((l >> 4) & 1) | (q << 1);
      py = 16 * w + d3; px = 16 * e1 + e3;
    } else {
      const int e1 = l & 3, e2 = (l >> 2) & 3, d2 = ((l >> 4) & 1) | (q << 1);
      py = 16 * w + 4 * d2; px = 16 * e1 + 4 * e2;
    }
  }
};

// Frequency index of storage row/column after the three forward passes:
// k = d0 + R0*d1 + R0*R1*d2 (digit reversal of the storage index).
template <class C>
__device__ __forceinline__ int freq_y(int py) {
  return py / C::sy(0) + C::ry(0) * ((py / C::sy(1)) % C::ry(1)) + C::ry(0) * C::ry(1) * (py % C::ry(2));
}
template <class C>
__device__ __forceinline__ int freq_x(int px) {
  return px / C::sx(0) + C::rx(0) * ((px / C::sx(1)) % C::rx(1)) + C::rx(0) * C::rx(1) * (px % C::rx(2));
}

template <class C, int J>
struct PassShape {
  static constexpr int RY = C::ry(J), RX = C::rx(J), G = RY * RX, Q = C::V / G;
  static constexpr int SY = C::sy(J), SX = C::sx(J);
  static_assert(Q * G == C::V, "group size must divide the per-thread count");
};

// Launder a value through an empty asm so index arithmetic derived from it
// is recomputed where it is used instead of being hoisted out of the slice
// loop and pinned in registers.
__device__ __forceinline__ int opaque(int x) {
  asm volatile("" : "+r"(x));
  return x;
}

template <class C, int J>
__device__ __forceinline__ void xch_store(const float2 (&v)[C::V], float2* sm, int t) {
  using P = PassShape<C, J>;
  t = opaque(t);
  static_for<0, P::Q>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    int py, px;
    C::template base<J>(t, q, py, px);
    static_for<0, P::RY>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      static_for<0, P::RX>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        sm[(py + a * P::SY) * C::M + C::swz(px + b * P::SX)] = v[q * P::G + a * P::RX + b];
      });
    });
  });
}

template <class C, int J>
__device__ __forceinline__ void xch_load(float2 (&v)[C::V], const float2* sm, int t) {
  using P = PassShape<C, J>;
  t = opaque(t);
  static_for<0, P::Q>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    int py, px;
    C::template base<J>(t, q, py, px);
    static_for<0, P::RY>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      static_for<0, P::RX>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        v[q * P::G + a * P::RX + b] = sm[(py + a * P::SY) * C::M + C::swz(px + b * P::SX)];
      });
    });
  });
}

// One radix pass on the registers.  Forward: DFT over digit J of y (for every
// x element), DFT over digit J of x (for every y element), then the twiddle
// w_M^(ey*a' + ex*b') that couples digit J to the lower digits.  Inverse: the
// conjugate twiddle, then the inverse DFTs (exact inverse up to the factor RY*RX).
// FACT selects factored twiddles w^(ey a) * w^(ex b): fewer table reads but
// one more rounding per element.  The forward model (whose rounding the
// amplitude residual amplifies) uses exact table values; the adjoint, which
// is linear in the residual, uses the factored form.
template <class C, int J, bool INV, bool FACT = false>
__device__ __forceinline__ void pass_compute(float2 (&v)[C::V], const float2* __restrict__ tw, int t) {
  using P = PassShape<C, J>;
  t = opaque(t);
  static_for<0, P::Q>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    constexpr int o = q * P::G;
    [[maybe_unused]] int ey = 0, ex = 0;
    if constexpr (J < 2) {
      int py, px;
      C::template base<J>(t, q, py, px);
      ey = (C::M / (P::RY * P::SY)) * (py & (P::SY - 1));
      ex = (C::M / (P::RX * P::SX)) * (px & (P::SX - 1));
    }
    auto twiddle = [&]() {
      if constexpr (J < 2 && FACT) {
        // w^(ey a + ex b) = w^(ey a) * w^(ex b): RY-1 + RX-1 table reads and
        // one extra product per element with a, b > 0.
        float2 txv[P::RX];
        static_for<1, P::RX>([&](auto bb) {
          constexpr int b = decltype(bb)::value;
          txv[b] = tw[(ex * b) & (C::M - 1)];
        });
        static_for<0, P::RY>([&](auto aa) {
          constexpr int a = decltype(aa)::value;
          float2 ty = make_float2(1.f, 0.f);
          if constexpr (a != 0) ty = tw[(ey * a) & (C::M - 1)];
          static_for<0, P::RX>([&](auto bb) {
            constexpr int b = decltype(bb)::value;
            if constexpr (a != 0 && b != 0) {
              v[o + a * P::RX + b] = cmul_opt<INV>(v[o + a * P::RX + b], cmul(ty, txv[b]));
            } else if constexpr (a != 0) {
              v[o + a * P::RX + b] = cmul_opt<INV>(v[o + a * P::RX + b], ty);
            } else if constexpr (b != 0) {
              v[o + a * P::RX + b] = cmul_opt<INV>(v[o + a * P::RX + b], txv[b]);
            }
          });
        });
      } else if constexpr (J < 2) {
        static_for<0, P::RY>([&](auto aa) {
          constexpr int a = decltype(aa)::value;
          static_for<0, P::RX>([&](auto bb) {
            constexpr int b = decltype(bb)::value;
            if constexpr (a != 0 || b != 0) {
              const float2 w = tw[(ey * a + ex * b) & (C::M - 1)];
              v[o + a * P::RX + b] = cmul_opt<INV>(v[o + a * P::RX + b], w);
            }
          });
        });
      }
    };
    if constexpr (INV) twiddle();
    static_for<0, P::RX>([&](auto bb) {
      constexpr int b = decltype(bb)::value;
      dft_at<P::RY, INV, o + b, P::RX>(v);
    });
    static_for<0, P::RY>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      dft_at<P::RX, INV, o + a * P::RX, 1>(v);
    });
    if constexpr (!INV) twiddle();
  });
}

// registers in pass-0 grouping (natural storage) -> unnormalised forward DFT,
// registers in pass-2 grouping (digit-reversed storage)
template <class C, bool FACT = false>
__device__ __forceinline__ void fft_fwd(float2 (&v)[C::V], float2* sm, const float2* tw, int t) {
  pass_compute<C, 0, false, FACT>(v, tw, t);
  xch_store<C, 0>(v, sm, t);
  __syncthreads();
  xch_load<C, 1>(v, sm, t);
  pass_compute<C, 1, false, FACT>(v, tw, t);
  xch_store<C, 1>(v, sm, t);
  C::sync12(t);
  xch_load<C, 2>(v, sm, t);
  pass_compute<C, 2, false, FACT>(v, tw, t);
}

// exact reverse of fft_fwd: unnormalised inverse DFT (times M*M relative to
// the true inverse), registers back in pass-0 grouping
template <class C, bool FACT = false>
__device__ __forceinline__ void fft_inv(float2 (&v)[C::V], float2* sm, const float2* tw, int t) {
  pass_compute<C, 2, true, FACT>(v, tw, t);
  xch_store<C, 2>(v, sm, t);
  C::sync12(t);
  xch_load<C, 1>(v, sm, t);
  pass_compute<C, 1, true, FACT>(v, tw, t);
  xch_store<C, 1>(v, sm, t);
  __syncthreads();
  xch_load<C, 0>(v, sm, t);
  pass_compute<C, 0, true, FACT>(v, tw, t);
}

// Multiply the spectrum (pass-2 grouping) by h(ky)*h(kx) (or its conjugate);
// hs[k] holds one separable factor of the propagator in FFT order.
template <class C, bool CONJ>
__device__ __forceinline__ void mul_separable(float2 (&v)[C::V], const float2* __restrict__ hs, int t) {
  using P = PassShape<C, 2>;
  t = opaque(t);
  static_for<0, P::Q>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    int py, px;
    C::template base<2>(t, q, py, px);
    const int ky0 = freq_y<C>(py), kx0 = freq_x<C>(px);
    float2 hx[P::RX];
    static_for<0, P::RX>([&](auto bb) {
      constexpr int b = decltype(bb)::value;
      hx[b] = hs[kx0 + C::rx(0) * C::rx(1) * b];
    });
    static_for<0, P::RY>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      const float2 hy = hs[ky0 + C::ry(0) * C::ry(1) * a];
      static_for<0, P::RX>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        const float2 hh = cmul(hy, hx[b]);
        v[q * P::G + a * P::RX + b] = cmul_opt<CONJ>(v[q * P::G + a * P::RX + b], hh);
      });
    });
  });
}

// Multiply the spectrum (pass-2 grouping) by the propagator read from a full
// M x M table h2[ky][kx] (FFT order), each entry rounded once from FP64: one
// rounding per element fewer than forming h(ky) h(kx) here.  The table is
// read through the read-only cache (the same 64 or 128 KiB for every block).
template <class C, bool CONJ>
__device__ __forceinline__ void mul_table(float2 (&v)[C::V], const float2* __restrict__ h2, int t) {
  using P = PassShape<C, 2>;
  t = opaque(t);
  static_for<0, P::Q>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    int py, px;
    C::template base<2>(t, q, py, px);
    const float2* hp = h2 + freq_y<C>(py) * C::M + freq_x<C>(px);
    float2 hh[P::G];
    static_for<0, P::RY>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      static_for<0, P::RX>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        hh[a * P::RX + b] = __ldg(hp + a * C::ry(0) * C::ry(1) * C::M + b * C::rx(0) * C::rx(1));
      });
    });
    static_for<0, P::G>([&](auto ee) {
      constexpr int e = decltype(ee)::value;
      v[q * P::G + e] = cmul_opt<CONJ>(v[q * P::G + e], hh[e]);
    });
  });
}

}  // namespace ptycho
