// Device code of the transforms along the homogeneous direction (Table 1): the half-length
// complex FFT (mixed-radix Stockham), the real-to-real pre- and post-processing, and the forward
// transform of one chunk of columns. Included by the transform kernels (kern_transform.cu) and by
// the fused forward transform + on-chip solve (kern_bottom.cu); everything here is in an unnamed
// namespace, so each translation unit has its own copy.
#pragma once

#include "kern_common.cuh"
#include "snac_impl.h"

namespace snac {
namespace {

template <typename T>
struct Cx {
  T re, im;
};
template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ Cx<T> conj(Cx<T> a) {
  return {a.re, -a.im};
}

// FP64 <-> FP32 conversions by integer operations on the bit patterns. GB300 runs the hardware
// conversions on its FP64 pipe (2 lanes per clock per multiprocessor), where they cost as much as
// the transforms' FP64 arithmetic; these use the integer pipes instead.
//   to_f32: round to nearest even; |x| below the FP32 normal range gives a signed zero, above it (and
//           Inf) a signed infinity, NaN a NaN.
//   to_f64: exact for normal floats and infinities/NaN; FP32 subnormals (below 1.2e-38) give a
//           signed zero.
__device__ __forceinline__ float to_f32(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned sign = hw & 0x80000000u;
  const int e11 = (int)((hw >> 20) & 0x7ffu);
  const int e8 = e11 - 896;  // FP32 exponent field
  // mantissa: top 23 of the 52 bits, then the round bit and whether any lower bit is set
  unsigned m = ((hw & 0x000fffffu) << 3) | (lw >> 29);
  const unsigned rest = lw & 0x1fffffffu;
  const bool up = (rest > 0x10000000u) || (rest == 0x10000000u && (m & 1u));
  unsigned bits = ((unsigned)e8 << 23) + m + (up ? 1u : 0u);  // a mantissa carry moves into the exponent
  if (e8 <= 0) bits = 0u;                                     // below the normal range (and zero)
  if (e8 >= 255 || bits >= 0x7f800000u) bits = 0x7f800000u;  // overflow and Inf
  if (e11 == 0x7ff && ((hw & 0x000fffffu) | lw)) bits = 0x7fc00000u;  // NaN
  return __uint_as_float(bits | sign);
}

__device__ __forceinline__ double to_f64(float y) {
  const unsigned b = __float_as_uint(y);
  const unsigned sign = b & 0x80000000u;
  const unsigned e8 = (b >> 23) & 0xffu;
  const unsigned m = b & 0x007fffffu;
  unsigned hw = sign | ((e8 + 896u) << 20) | (m >> 3);
  unsigned lw = m << 29;
  if (e8 == 0u) hw = sign, lw = 0u;                      // zero (and subnormals)
  if (e8 == 255u) hw = sign | 0x7ff00000u | (m >> 3);    // Inf and NaN
  return __hiloint2double((int)hw, (int)lw);
}

template <typename T, typename TI>
__device__ __forceinline__ T to_inner(TI v) {
  if constexpr (sizeof(T) == 4 && sizeof(TI) == 8) return to_f32(v);
  else return (T)v;
}

template <typename T>
__device__ __forceinline__ double to_double(T v) {
  if constexpr (sizeof(T) == 4) return to_f64(v);
  else return v;
}

template <typename T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) {
  return {a.re + b.re, a.im + b.im};
}

// Work split of a transform CTA of NT threads over a chunk of TC columns (NT a multiple of TC):
// thread t keeps column t % TC in every pass and takes rows t / TC, t / TC + NT / TC, ... of it,
// so column offsets and pointers are set up once per thread, not per element.
template <int TC, int NT>
__device__ __forceinline__ int my_col() {
  static_assert(NT % TC == 0, "a transform CTA covers whole rows of its chunk");
  return threadIdx.x % TC;
}
template <int TC, int NT>
__device__ __forceinline__ int my_row() {
  return threadIdx.x / TC;
}

// One Stockham stage of radix R on TC columns: groups of R consecutive length-Ls transforms are
// merged into transforms of length R Ls. Input of group j, point k: a_p = x[(j + p r) Ls + k] times
// the twiddle w^(p k r) (w = exp(-2 pi i / m), r = m / (R Ls)); outputs y_q = sum_p a_p omega_R^(p q)
// at (R j + q) Ls + k, with omega_R^s = w^(s m / R) taken from the same table. Radices 3 and 5 are
// unrolled; any other prime goes through the runtime-radix stage below (O(R) work per point).
template <typename T, int TC, int NT, int R>
__device__ void stage_r(const Cx<T>* __restrict__ X, Cx<T>* __restrict__ Y, int m, int Ls,
                        const Cx<T>* __restrict__ tw, bool inverse) {
  const int r = m / (R * Ls), mr = m / R;
  const int c = my_col<TC, NT>();
  for (int t = my_row<TC, NT>(); t < m / R; t += NT / TC) {
    const int j = t / Ls, k = t - j * Ls;
    Cx<T> a[R];
#pragma unroll
    for (int p = 0; p < R; ++p) {
      a[p] = X[((j + p * r) * Ls + k) * TC + c];
      if (p > 0 && k > 0) {
        Cx<T> w = tw[p * k * r];
        if (inverse) w.im = -w.im;
        a[p] = cmul(w, a[p]);
      }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      Cx<T> acc = a[0];
#pragma unroll
      for (int p = 1; p < R; ++p) {
        Cx<T> w = tw[((p * q) % R) * mr];
        if (inverse) w.im = -w.im;
        acc = cadd(acc, cmul(w, a[p]));
      }
      Y[((R * j + q) * Ls + k) * TC + c] = acc;
    }
  }
  __syncthreads();
}

// The same stage for a radix known only at run time (a prime factor above 5): one output per
// thread and iteration, y = sum_p w^(p k r + (p q mod R) m / R) x_p.
template <typename T, int TC, int NT>
__device__ void stage_any(const Cx<T>* __restrict__ X, Cx<T>* __restrict__ Y, int m, int Ls, int R,
                          const Cx<T>* __restrict__ tw, bool inverse) {
  const int r = m / (R * Ls), mr = m / R;
  const int c = my_col<TC, NT>();
  for (int o = my_row<TC, NT>(); o < m; o += NT / TC) {
    const int k = o % Ls, q = (o / Ls) % R, j = o / (Ls * R);
    Cx<T> acc = {0, 0};
    for (int p = 0; p < R; ++p) {
      const int e = (int)(((long long)p * k * r + (long long)((p * q) % R) * mr) % m);
      Cx<T> w = tw[e];
      if (inverse) w.im = -w.im;
      acc = cadd(acc, cmul(w, X[((j + p * r) * Ls + k) * TC + c]));
    }
    Y[o * TC + c] = acc;
  }
  __syncthreads();
}

// Complex DFT of length m of TC columns held as buf[j * TC + c]. Forward: exp(-2 pi i jk/m);
// inverse (unnormalised): exp(+2 pi i jk/m). Returns the buffer holding the result.
// Stockham autosort, mixed radix: the factors 4 (with the exact rotations by +-i) and 2 first, while
// the merged length Ls is a power of two; then 3, 5 and any remaining prime.
template <typename T, int TC, int NT>
__device__ Cx<T>* cfft(Cx<T>* X, Cx<T>* Y, int m, const Cx<T>* __restrict__ tw, bool inverse) {
  if (m == 1) return X;
  const int c = my_col<TC, NT>();
  int Ls = 1;
  {
    // Merge groups of four length-Ls transforms into length-4Ls transforms while four remain
    // (radix 4: three twiddle products per four points), then pairs (radix 2) once if a factor 2
    // is left. Output stage q of a group: y_q = sum_p (w^(p k) x_p) omega_4^(p q).
    int lg = 0;
    for (; (m / Ls) % 4 == 0; Ls <<= 2, lg += 2) {
      const int r = m / (4 * Ls);
      for (int t = my_row<TC, NT>(); t < m / 4; t += NT / TC) {
        const int j = t >> lg, k = t & (Ls - 1);
        const Cx<T>* x = X + (j * Ls + k) * TC + c;
        const int sx = r * Ls * TC;
        Cx<T> a0 = x[0];
        Cx<T> a1 = x[sx];
        Cx<T> a2 = x[2 * sx];
        Cx<T> a3 = x[3 * sx];
        if (Ls > 1) {  // the first stage has k = 0 only: unit twiddles
          Cx<T> w1 = tw[k * r], w2 = tw[2 * k * r], w3 = tw[3 * k * r];
          if (inverse) {
            w1.im = -w1.im;
            w2.im = -w2.im;
            w3.im = -w3.im;
          }
          a1 = cmul(w1, a1);
          a2 = cmul(w2, a2);
          a3 = cmul(w3, a3);
        }
        const Cx<T> s02 = {a0.re + a2.re, a0.im + a2.im}, d02 = {a0.re - a2.re, a0.im - a2.im};
        const Cx<T> s13 = {a1.re + a3.re, a1.im + a3.im}, d13 = {a1.re - a3.re, a1.im - a3.im};
        // omega_4 d13: -i d13 forward, +i d13 inverse
        const Cx<T> od = inverse ? Cx<T>{-d13.im, d13.re} : Cx<T>{d13.im, -d13.re};
        Cx<T>* y = Y + (4 * j * Ls + k) * TC + c;
        const int sy = Ls * TC;
        y[0] = {s02.re + s13.re, s02.im + s13.im};
        y[sy] = {d02.re + od.re, d02.im + od.im};
        y[2 * sy] = {s02.re - s13.re, s02.im - s13.im};
        y[3 * sy] = {d02.re - od.re, d02.im - od.im};
      }
      __syncthreads();
      Cx<T>* s = X;
      X = Y;
      Y = s;
    }
    for (; (m / Ls) % 2 == 0; Ls <<= 1, ++lg) {
      const int r = m / (2 * Ls);
      for (int t = my_row<TC, NT>(); t < m / 2; t += NT / TC) {
        const int j = t >> lg, k = t & (Ls - 1);
        Cx<T> w = tw[k * r];
        if (inverse) w.im = -w.im;
        const Cx<T> a = X[(j * Ls + k) * TC + c];
        const Cx<T> b = cmul(w, X[((j + r) * Ls + k) * TC + c]);
        Y[(2 * j * Ls + k) * TC + c] = {a.re + b.re, a.im + b.im};
        Y[(2 * j * Ls + Ls + k) * TC + c] = {a.re - b.re, a.im - b.im};
      }
      __syncthreads();
      Cx<T>* s = X;
      X = Y;
      Y = s;
    }
  }
  auto swap = [&]() {
    Cx<T>* s = X;
    X = Y;
    Y = s;
  };
  for (; (m / Ls) % 3 == 0; Ls *= 3) {
    stage_r<T, TC, NT, 3>(X, Y, m, Ls, tw, inverse);
    swap();
  }
  for (; (m / Ls) % 5 == 0; Ls *= 5) {
    stage_r<T, TC, NT, 5>(X, Y, m, Ls, tw, inverse);
    swap();
  }
  for (int p = 7; Ls < m; p += 2) {
    for (; (m / Ls) % p == 0; Ls *= p) {
      stage_any<T, TC, NT>(X, Y, m, Ls, p, tw, inverse);
      swap();
    }
  }
  return X;
}

template <typename T>
struct Tw {
  const Cx<T>* fft;
  const Cx<T>* twn;
  const Cx<T>* tw2n;
  const Cx<T>* tw4a;
  const Cx<T>* tw4b;
};

// X_k (k = 0..m) of the real DFT of the length-n sequence packed as Z = FFT_m(x_2j + i x_2j+1).
template <typename T, int TC>
__device__ __forceinline__ Cx<T> rdft_bin(const Cx<T>* R, int k, int m, int c, const Tw<T>& tw) {
  const Cx<T> zk = R[(k == m ? 0 : k) * TC + c];
  const Cx<T> zc = conj(R[(k == 0 ? 0 : m - k) * TC + c]);
  const Cx<T> E = {(T)0.5 * (zk.re + zc.re), (T)0.5 * (zk.im + zc.im)};
  const Cx<T> d = {zk.re - zc.re, zk.im - zc.im};
  const Cx<T> O = {(T)0.5 * d.im, (T)-0.5 * d.re};  // d / (2i)
  const Cx<T> wo = cmul(tw.twn[k], O);
  return {E.re + wo.re, E.im + wo.im};
}

// Z_k (k < m) for the inverse real DFT, from half-complex bins X_k and conj(X_{m-k}).
template <typename T>
__device__ __forceinline__ Cx<T> irdft_pre(Cx<T> xk, Cx<T> xmk, const Cx<T>& twn_k) {
  const Cx<T> xc = conj(xmk);
  const Cx<T> E = {xk.re + xc.re, xk.im + xc.im};
  const Cx<T> O = cmul({xk.re - xc.re, xk.im - xc.im}, conj(twn_k));
  return {E.re - O.im, E.im + O.re};  // E + i O
}

// Loads from HBM per thread in flight before their first use: the column loads of a chunk are
// independent, and issuing them in batches keeps enough bytes in flight to cover the DRAM latency.
constexpr int LBATCH = 8;

// Caller offsets (at k = 0) of the chunk's columns, and the caller stride along the homogeneous axis.
template <int TC>
__device__ __forceinline__ long long chunk_columns(const ChunkDev& ch, const BlockDev& B, const CallerBlk* __restrict__ cb,
                                                   long long (&coff)[TC]) {
  const CallerBlk C = cb[ch.b];
  if (threadIdx.x < TC) {
    const long long pc = (long long)ch.c0 + threadIdx.x;  // plane cell of the block
    coff[threadIdx.x] = C.off3 + (pc % B.nx) * C.s[0] + (pc / B.nx) * C.s[1];
  }
  __syncthreads();
  return C.s[2];
}

// Forward transform of one chunk by a CTA of NT threads (dynamic shared memory: two buffers of
// n/2 x TC complex values). The loads go straight into the half-length FFT's input for the kinds
// whose reordering is a pure permutation (PP, NN, DD: z_j = v_2j + i v_2j+1 with v = x (PP) or
// Makhoul's v_t = x_2t (t < m), x_2(n-1-t)+1 (t >= m)); DCT-IV / DST-IV need a twiddled pre-pass.
// The sign flip of the DST kinds ((-1)^k x_k) is applied as the values arrive.
template <typename T, int TC, int KIND, typename TI, int NT>
__device__ void forward_chunk(const ChunkDev ch, const BlockDev* __restrict__ blk, const CallerBlk* __restrict__ cb,
                              int n, const Tw<T>& tw, const TI* __restrict__ in3, T* __restrict__ out, long long ncell,
                              T sub0, int split, unsigned char* smem) {
  constexpr int kind = KIND;
  constexpr int RS = NT / TC;  // rows per pass
  constexpr bool direct = kind == KIND_PP || kind == KIND_NN || kind == KIND_DD;
  constexpr bool flip = kind == KIND_DD || kind == KIND_DN;
  __shared__ long long coff[TC];
  __shared__ long long ooff[TC];  // position of each column in a mode plane (plain or colour-split)
  const int m = n / 2;
  Cx<T>* A = reinterpret_cast<Cx<T>*>(smem);
  Cx<T>* Bf = A + m * TC;
  T* xs = reinterpret_cast<T*>(Bf);  // n x TC reals, aliases Bf (DCT-IV / DST-IV only)
  T* Af = reinterpret_cast<T*>(A);
  const BlockDev B = blk[ch.b];
  if (threadIdx.x < TC) {
    const int pc = ch.c0 + threadIdx.x;
    ooff[threadIdx.x] = split ? split_cell(B, pc % B.nx, pc / B.nx) : B.off + pc;
  }
  const long long sk = chunk_columns<TC>(ch, B, cb, coff);  // (its barrier also covers ooff)
  const int c = my_col<TC, NT>(), r0 = my_row<TC, NT>();
  const bool live = c < ch.ncol;
  // x_k of column cc, as it arrives
  auto store = [&](int k, int cc, TI v) {
    T x = to_inner<T, TI>(v);
    if (flip && (k & 1)) x = -x;
    if constexpr (direct) {
      const int t = kind == KIND_PP ? k : ((k & 1) ? n - 1 - (k >> 1) : (k >> 1));
      Af[(((t >> 1) * TC + cc) << 1) + (t & 1)] = x;
    } else {
      xs[k * TC + cc] = x;
    }
  };
  if (sk != 1) {  // rows of the chunk are TC consecutive cells (coalesced); column c is this thread's
    const TI* src = in3 + (live ? coff[c] : 0);
    for (int k0 = r0; k0 < n; k0 += LBATCH * RS) {
      TI v[LBATCH];
#pragma unroll
      for (int u = 0; u < LBATCH; ++u) {
        const int k = k0 + u * RS;
        v[u] = live && k < n ? src[(long long)k * sk] : (TI)0;
      }
#pragma unroll
      for (int u = 0; u < LBATCH; ++u) {
        const int k = k0 + u * RS;
        if (k < n) store(k, c, v[u]);
      }
    }
  } else {  // the homogeneous axis is the caller's contiguous one: consecutive threads run along it
    for (int i0 = threadIdx.x; i0 < n * TC; i0 += LBATCH * NT) {
      TI v[LBATCH];
#pragma unroll
      for (int u = 0; u < LBATCH; ++u) {
        const int idx = i0 + u * NT;
        const int k = idx % n, cc = idx / n;
        v[u] = idx < n * TC && cc < ch.ncol ? in3[coff[cc] + k] : (TI)0;
      }
#pragma unroll
      for (int u = 0; u < LBATCH; ++u) {
        const int idx = i0 + u * NT;
        if (idx < n * TC) store(idx % n, idx / n, v[u]);
      }
    }
  }
  __syncthreads();
  if constexpr (!direct) {  // t_j = (x_2j + i x_{n-1-2j}) e^{-i pi (4j+1)/4n}
    for (int j = r0; j < m; j += RS) A[j * TC + c] = cmul(Cx<T>{xs[2 * j * TC + c], xs[(n - 1 - 2 * j) * TC + c]}, tw.tw4a[j]);
    __syncthreads();
  }
  const Cx<T>* R = cfft<T, TC, NT>(A, Bf, m, tw.fft, false);
  // F(x - shift0) = F(x) - shift0 F(1); F(1) is zero outside mode 0
  T* ob = out + (live ? ooff[c] : 0);
  auto put = [&](int q, T y) {
    if (q == 0) y -= sub0;
    if (live) ob[(long long)q * ncell] = y;
  };
  if constexpr (direct) {
    // each half-spectrum bin k = 0..m once; it gives output k and its mirror n - k
    for (int k = r0; k <= m; k += RS) {
      const Cx<T> X = rdft_bin<T, TC>(R, k, m, c, tw);
      const bool mirror = k > 0 && k < m;
      if (kind == KIND_PP) {
        put(k, X.re);
        if (mirror) put(n - k, X.im);
      } else {
        const Cx<T> w = tw.tw2n[k];
        const T y = (T)2 * (w.re * X.re - w.im * X.im);
        put(kind == KIND_DD ? n - 1 - k : k, y);
        if (mirror) {  // bin n - k is conj(X_k)
          const Cx<T> wm = tw.tw2n[n - k];
          const T ym = (T)2 * (wm.re * X.re + wm.im * X.im);
          put(kind == KIND_DD ? k - 1 : n - k, ym);
        }
      }
    }
  } else {
    for (int q = r0; q < n; q += RS) {
      const int qq = kind == KIND_DN ? n - 1 - q : q;
      T y;
      if ((qq & 1) == 0) {
        const int k = qq / 2;
        y = (T)2 * cmul(R[k * TC + c], tw.tw4b[k]).re;
      } else {
        const int k = (n - 1 - qq) / 2;
        y = (T)-2 * cmul(R[k * TC + c], tw.tw4b[k]).im;
      }
      put(q, y);
    }
  }
}

}  // namespace
}  // namespace snac
