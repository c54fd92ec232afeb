// Real-to-real transforms along the homogeneous direction (Table 1; Algorithm 1, first and third
// loops), batched over x-y columns. One CTA transforms TC consecutive columns of one block: the
// columns are loaded row by row (coalesced along x), reordered into a complex sequence of half
// length m = n/2, transformed by a shared-memory complex FFT (mixed-radix Stockham: radices 4, 2,
// 3, 5 and any other prime factor), and post-processed into the real output. Twiddles come from host-built
// tables; the kernels evaluate no transcendental function.
//
// Reductions to a half-length complex FFT (conventions of the unnormalised real-to-real
// transforms, theta of Table 1):
//   PP  real DFT in half-complex order: z_j = x_2j + i x_2j+1, split the spectrum into the even and
//       odd halves (Cooley-Tukey); the inverse runs the same steps backwards.
//   NN  DCT-II by Makhoul's reordering v = (x_0, x_2, ..., x_3, x_1), Y_k = 2 Re(e^{-i pi k/2n} V_k)
//       with V the real DFT of v; DCT-III inverts it.
//   DD  DST-II_k(x) = DCT-II_{n-1-k}((-1)^j x_j); DST-III(X)_j = (-1)^j DCT-III(X reversed)_j.
//   ND  DCT-IV: t_j = (x_2j + i x_{n-1-2j}) e^{-i pi (4j+1)/4n}, T = FFT_m(t), c_k = T_k e^{-i pi k/n},
//       Y_2k = 2 Re c_k, Y_{n-1-2k} = -2 Im c_k. It is its own inverse (x 2n).
//   DN  DST-IV_k(x) = DCT-IV_{n-1-k}((-1)^j x_j), its own inverse (x 2n).
#include <cmath>

#include "transform_dev.cuh"

namespace snac {
namespace {

// One CTA of TNT threads per chunk of TC columns.
constexpr int TNT = 256;

template <typename T, int TC, int KIND, typename TI>
__global__ void __launch_bounds__(TNT, 3) k_forward(const ChunkDev* __restrict__ chunks, const BlockDev* __restrict__ blk,
                                                 const CallerBlk* __restrict__ cb, int n, Tw<T> tw,
                                                 const TI* __restrict__ in3, T* __restrict__ out, long long ncell,
                                                 T sub0, int split) {
  extern __shared__ __align__(16) unsigned char smem[];
  forward_chunk<T, TC, KIND, TI, TNT>(chunks[blockIdx.x], blk, cb, n, tw, in3, out, ncell, sub0, split, smem);
}

template <typename T, int TC, int KIND>
__global__ void __launch_bounds__(TNT, 3) k_backward(const ChunkDev* __restrict__ chunks, const BlockDev* __restrict__ blk,
                                                  const CallerBlk* __restrict__ cb, int n, Tw<T> tw,
                                                  const T* __restrict__ modes, double* __restrict__ p3, long long ncell,
                                                  double inv_theta) {
  constexpr int kind = KIND;
  constexpr int RS = TNT / TC;  // rows per pass
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = n / 2;
  Cx<T>* A = reinterpret_cast<Cx<T>*>(smem);
  Cx<T>* Bf = A + m * TC;
  T* xs = reinterpret_cast<T*>(Bf);
  const ChunkDev ch = chunks[blockIdx.x];
  const BlockDev B = blk[ch.b];
  const int c = my_col<TC, TNT>(), r0 = my_row<TC, TNT>();
  const bool live = c < ch.ncol;
  {
    const T* src = modes + B.off + ch.c0 + (live ? c : 0);
    for (int q0 = r0; q0 < n; q0 += LBATCH * RS) {
      T v[LBATCH];
#pragma unroll
      for (int u = 0; u < LBATCH; ++u) {
        const int q = q0 + u * RS;
        v[u] = live && q < n ? src[(long long)q * ncell] : (T)0;
      }
#pragma unroll
      for (int u = 0; u < LBATCH; ++u) {
        const int q = q0 + u * RS;
        if (q < n) xs[q * TC + c] = v[u];
      }
    }
  }
  __syncthreads();
  const bool rev = kind == KIND_DD;                 // DST-III reads X reversed
  const bool flip = kind == KIND_DN;                // DST-IV = DCT-IV of the sign-flipped input, reversed
  auto X = [&](int k) -> T {
    if (k >= n) return (T)0;
    const int kk = rev ? n - 1 - k : k;
    const T v = xs[kk * TC + c];
    return (flip && (k & 1)) ? -v : v;
  };
  if (kind == KIND_PP || kind == KIND_NN || kind == KIND_DD) {
    // half-spectrum bin j of the real DFT being inverted: PP the stored bins (X_j, X_{n-j}),
    // NN/DD V_j = e^{+i pi j/2n} (X_j - i X_{n-j}) (the real DFT of the reordered sequence)
    auto bin = [&](int j) -> Cx<T> {
      if (kind == KIND_PP) return (j == 0 || j == m) ? Cx<T>{X(j), 0} : Cx<T>{X(j), X(n - j)};
      Cx<T> v = cmul(conj(tw.tw2n[j]), Cx<T>{X(j), -X(n - j)});
      if (j == 0 || j == m) v.im = 0;
      return v;
    };
    // z_k needs bins k and m - k: each pair once, giving z_k and z_{m-k}
    for (int k = r0; k < m / 2 + 1; k += RS) {
      const Cx<T> b1 = bin(k), b2 = bin(m - k);
      A[k * TC + c] = irdft_pre(b1, b2, tw.twn[k]);
      if (k > 0 && m - k != k) A[(m - k) * TC + c] = irdft_pre(b2, b1, tw.twn[m - k]);
    }
  } else {
    for (int k = r0; k < m; k += RS) A[k * TC + c] = cmul(Cx<T>{X(2 * k), X(n - 1 - 2 * k)}, tw.tw4a[k]);
  }
  __syncthreads();
  const bool inv = kind == KIND_PP || kind == KIND_NN || kind == KIND_DD;
  const Cx<T>* R = cfft<T, TC, TNT>(A, Bf, m, tw.fft, inv);
  __shared__ long long coff[TC];
  const long long sk = chunk_columns<TC>(ch, B, cb, coff);
  // output j of column cc
  auto y_of = [&](int j, int cc) -> T {
    T y;
    if (kind == KIND_PP) {
      const Cx<T> z = R[(j >> 1) * TC + cc];
      y = (j & 1) ? z.im : z.re;
    } else if (kind == KIND_NN || kind == KIND_DD) {
      const int t = (j & 1) ? n - 1 - (j >> 1) : (j >> 1);  // x_2t = v_t, x_2t+1 = v_{n-1-t}
      const Cx<T> z = R[(t >> 1) * TC + cc];
      y = (t & 1) ? z.im : z.re;
      if (kind == KIND_DD && (j & 1)) y = -y;
    } else {
      const int qq = kind == KIND_DN ? n - 1 - j : j;
      if ((qq & 1) == 0) {
        const int k = qq / 2;
        y = (T)2 * cmul(R[k * TC + cc], tw.tw4b[k]).re;
      } else {
        const int k = (n - 1 - qq) / 2;
        y = (T)-2 * cmul(R[k * TC + cc], tw.tw4b[k]).im;
      }
    }
    return y;
  };
  // p += y / theta: the old values of a batch are loaded before any of them is written back
  if (sk != 1) {  // column c is this thread's
    double* dst = p3 + (live ? coff[c] : 0);
    for (int j0 = r0; j0 < n; j0 += LBATCH * RS) {
      double old[LBATCH];
#pragma unroll
      for (int u = 0; u < LBATCH; ++u) {
        const int j = j0 + u * RS;
        old[u] = live && j < n ? dst[(long long)j * sk] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < LBATCH; ++u) {
        const int j = j0 + u * RS;
        if (j >= n) break;
        const T y = y_of(j, c);
        if (live) dst[(long long)j * sk] = fma(to_double(y), inv_theta, old[u]);
      }
    }
  } else {  // the homogeneous axis is the caller's contiguous one: consecutive threads run along it
    for (int i0 = threadIdx.x; i0 < n * TC; i0 += LBATCH * TNT) {
      double old[LBATCH];
#pragma unroll
      for (int u = 0; u < LBATCH; ++u) {
        const int idx = i0 + u * TNT;
        const int j = idx % n, cc = idx / n;
        old[u] = idx < n * TC && cc < ch.ncol ? p3[coff[cc] + j] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < LBATCH; ++u) {
        const int idx = i0 + u * TNT;
        if (idx >= n * TC) break;
        const int j = idx % n, cc = idx / n;
        const T y = y_of(j, cc);
        if (cc < ch.ncol) p3[coff[cc] + j] = fma(to_double(y), inv_theta, old[u]);
      }
    }
  }
}

// Dynamic shared memory of a transform launch: two half-length complex buffers of TC columns. The
// kernel's maximum is a function-wide attribute shared by every plan and thread, so it is always set
// to the largest need of any plan that uses this instantiation (128 KB: transform_columns keeps
// n_z x TC x 2 x sizeof(T) at or below it): a plan with a shorter axis never lowers it under a
// concurrent launch of a plan with a longer one.
template <typename T, int TC>
constexpr int kMaxSmem = 128 * 1024;

template <typename T>
Tw<T> make_tw(const snac_plan* P, const void* base) {
  const Cx<T>* t = reinterpret_cast<const Cx<T>*>(base);
  return Tw<T>{t + P->tw.fft, t + P->tw.twn, t + P->tw.tw2n, t + P->tw.tw4a, t + P->tw.tw4b};
}

// Where a transform's columns live: the block table and caller offsets/strides of the 3-D field,
// the cells of one mode plane of the output, and the field's cell count. The plan's own field, or a
// pencil of a sharded solve (one pseudo-block of ncols columns, [z][c] layout).
struct Geom {
  const BlockDev* blk;
  const CallerBlk* cb;
  long long ncell;
  double n3;
};

Geom plan_geom(const snac_plan* P) { return Geom{P->lev[0].d_blk, P->d_cblk, P->lev[0].ncell, (double)P->n3}; }

template <typename T, int TC, typename TI = double>
cudaError_t fwd_t(snac_plan* P, const Geom& G, const std::vector<ChunkDev>& ch, const ChunkDev* dch, const void* twb,
                  const TI* in3, void* modes, double shift0, bool split, cudaStream_t s) {
  // F(1) in mode 0: n for the real DFT (half-complex), 2n for the DCT-II; the other kinds have no
  // zero eigenvalue and are never shifted
  const double f1 = P->kind == KIND_PP ? (double)P->nzt : 2.0 * P->nzt;
  const T sub0 = (T)(shift0 * f1);
  const size_t smem = 2 * (size_t)(P->nzt / 2) * TC * sizeof(Cx<T>);
  const double n3 = G.n3;
  // read the 3-D field, write the modes; FFT model 2.5 log2(n) flops per point plus pre/post-processing
  LaunchScope ls(P, K_FORWARD, (double)(sizeof(TI) + sizeof(T)) * n3, (2.5 * std::log2((double)P->nzt) + 8.0) * n3, s);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem<T, TC>);
    kern<<<(unsigned)ch.size(), TNT, smem, s>>>(dch, G.blk, G.cb, P->nzt, make_tw<T>(P, twb), in3, (T*)modes, G.ncell,
                                                sub0, split ? 1 : 0);
  };
  switch (P->kind) {
    case KIND_PP: go(k_forward<T, TC, KIND_PP, TI>); break;
    case KIND_NN: go(k_forward<T, TC, KIND_NN, TI>); break;
    case KIND_DD: go(k_forward<T, TC, KIND_DD, TI>); break;
    case KIND_ND: go(k_forward<T, TC, KIND_ND, TI>); break;
    default: go(k_forward<T, TC, KIND_DN, TI>); break;
  }
  return cudaGetLastError();
}

template <typename T, int TC>
cudaError_t bwd_t(snac_plan* P, const Geom& G, const std::vector<ChunkDev>& ch, const ChunkDev* dch, const void* twb,
                  const void* modes, double* p3, double sign, cudaStream_t s) {
  const size_t smem = 2 * (size_t)(P->nzt / 2) * TC * sizeof(Cx<T>);
  const double n3 = G.n3;
  // read the modes, read and write the FP64 field
  LaunchScope ls(P, K_BACKWARD, (16.0 + sizeof(T)) * n3, (2.5 * std::log2((double)P->nzt) + 10.0) * n3, s);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem<T, TC>);
    kern<<<(unsigned)ch.size(), TNT, smem, s>>>(dch, G.blk, G.cb, P->nzt, make_tw<T>(P, twb), (const T*)modes, p3,
                                                G.ncell, sign / P->theta);
  };
  switch (P->kind) {
    case KIND_PP: go(k_backward<T, TC, KIND_PP>); break;
    case KIND_NN: go(k_backward<T, TC, KIND_NN>); break;
    case KIND_DD: go(k_backward<T, TC, KIND_DD>); break;
    case KIND_ND: go(k_backward<T, TC, KIND_ND>); break;
    default: go(k_backward<T, TC, KIND_DN>); break;
  }
  return cudaGetLastError();
}

}  // namespace

// The transform kernels are instantiated for the chunk widths transform_columns picks.
template <typename T, typename TI>
cudaError_t fwd_any(snac_plan* P, const Geom& G, const std::vector<ChunkDev>& ch, const ChunkDev* dch, const void* twb,
                    const TI* in3, void* modes, double shift0, bool split, cudaStream_t s) {
  const int tc = sizeof(T) == 8 ? P->tc64 : P->tc32;
  constexpr int B = sizeof(T) == 8 ? 8 : 16;
  if (tc == B) return fwd_t<T, B, TI>(P, G, ch, dch, twb, in3, modes, shift0, split, s);
  if (tc == B / 2) return fwd_t<T, B / 2, TI>(P, G, ch, dch, twb, in3, modes, shift0, split, s);
  if (tc == B / 4) return fwd_t<T, B / 4, TI>(P, G, ch, dch, twb, in3, modes, shift0, split, s);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t bwd_any(snac_plan* P, const Geom& G, const std::vector<ChunkDev>& ch, const ChunkDev* dch, const void* twb,
                    const void* modes, double* p3, double sign, cudaStream_t s) {
  const int tc = sizeof(T) == 8 ? P->tc64 : P->tc32;
  constexpr int B = sizeof(T) == 8 ? 8 : 16;
  if (tc == B) return bwd_t<T, B>(P, G, ch, dch, twb, modes, p3, sign, s);
  if (tc == B / 2) return bwd_t<T, B / 2>(P, G, ch, dch, twb, modes, p3, sign, s);
  if (tc == B / 4) return bwd_t<T, B / 4>(P, G, ch, dch, twb, modes, p3, sign, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_forward(snac_plan* P, const double* in3, void* modes, double shift0, bool split, cudaStream_t s) {
  if (shift0 != 0.0 && P->kind != KIND_PP && P->kind != KIND_NN) return cudaErrorInvalidValue;
  if (split && P->precision != SNAC_FP64) return cudaErrorInvalidValue;
  if (P->precision == SNAC_FP64)
    return fwd_any<double, double>(P, plan_geom(P), P->chunks64, P->d_chunks64, P->d_tw64, in3, modes, shift0, split, s);
  return fwd_any<float, double>(P, plan_geom(P), P->chunks32, P->d_chunks32, P->d_tw32, in3, modes, shift0, false, s);
}

cudaError_t launch_forward_f32(snac_plan* P, const float* in3, void* modes, cudaStream_t s) {
  if (P->precision != SNAC_MIXED) return cudaErrorInvalidValue;
  return fwd_any<float, float>(P, plan_geom(P), P->chunks32, P->d_chunks32, P->d_tw32, in3, modes, 0.0, false, s);
}

cudaError_t launch_backward_update(snac_plan* P, const void* modes, double* p3, cudaStream_t s, bool subtract) {
  const double sign = subtract ? -1.0 : 1.0;
  if (P->precision == SNAC_FP64)
    return bwd_any<double>(P, plan_geom(P), P->chunks64, P->d_chunks64, P->d_tw64, modes, p3, sign, s);
  return bwd_any<float>(P, plan_geom(P), P->chunks32, P->d_chunks32, P->d_tw32, modes, p3, sign, s);
}

// Pencil of a sharded solve: ncols columns stored [z][c], one pseudo-block (nx = ncols, ny = 1,
// caller strides 1, ncols, ncols), its chunk tables built on the first use of this width.
static cudaError_t pencil_tables(snac_plan* P, long long ncols) {
  if (P->pen_tcols == ncols) return cudaSuccess;
  for (void* p : P->pen_tallocs) cudaFree(p);
  P->pen_tallocs.clear();
  P->pen_tcols = -1;
  if (ncols < 1 || ncols >= (1LL << 31)) return cudaErrorInvalidValue;
  BlockDev b{};
  b.off = 0;
  b.nx = (int)ncols;
  b.ny = 1;
  for (int f = 0; f < 4; ++f) b.nbr[f] = -1;
  const CallerBlk c{0, {1, ncols, ncols}};
  P->pen_ch64.clear();
  P->pen_ch32.clear();
  const int t64 = P->tc64, t32 = P->tc32;
  for (long long c0 = 0; c0 < ncols; c0 += t64) P->pen_ch64.push_back({0, (int)c0, (int)std::min<long long>(t64, ncols - c0), 0});
  for (long long c0 = 0; c0 < ncols; c0 += t32) P->pen_ch32.push_back({0, (int)c0, (int)std::min<long long>(t32, ncols - c0), 0});
  auto put = [&](auto** d, const void* src, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc((void**)d, bytes);
    if (e != cudaSuccess) return e;
    P->pen_tallocs.push_back(*d);
    return cudaMemcpy(*d, src, bytes, cudaMemcpyHostToDevice);
  };
  cudaError_t e;
  if ((e = put(&P->d_pen_tblk, &b, sizeof b)) != cudaSuccess || (e = put(&P->d_pen_tcb, &c, sizeof c)) != cudaSuccess ||
      (e = put(&P->d_pen_ch64, P->pen_ch64.data(), P->pen_ch64.size() * sizeof(ChunkDev))) != cudaSuccess ||
      (e = put(&P->d_pen_ch32, P->pen_ch32.data(), P->pen_ch32.size() * sizeof(ChunkDev))) != cudaSuccess)
    return e;
  P->pen_tcols = ncols;
  return cudaSuccess;
}

cudaError_t launch_pencil_forward(snac_plan* P, long long ncols, const double* in, void* modes, cudaStream_t s) {
  cudaError_t e = pencil_tables(P, ncols);
  if (e != cudaSuccess) return e;
  const Geom G{P->d_pen_tblk, P->d_pen_tcb, ncols, (double)ncols * P->nzt};
  if (P->precision == SNAC_FP64)
    return fwd_any<double, double>(P, G, P->pen_ch64, P->d_pen_ch64, P->d_tw64, in, modes, 0.0, false, s);
  return fwd_any<float, double>(P, G, P->pen_ch32, P->d_pen_ch32, P->d_tw32, in, modes, 0.0, false, s);
}

cudaError_t launch_pencil_backward(snac_plan* P, long long ncols, const void* modes, double* p, cudaStream_t s) {
  cudaError_t e = pencil_tables(P, ncols);
  if (e != cudaSuccess) return e;
  const Geom G{P->d_pen_tblk, P->d_pen_tcb, ncols, (double)ncols * P->nzt};
  if (P->precision == SNAC_FP64)
    return bwd_any<double>(P, G, P->pen_ch64, P->d_pen_ch64, P->d_tw64, modes, p, 1.0, s);
  return bwd_any<float>(P, G, P->pen_ch32, P->d_pen_ch32, P->d_tw32, modes, p, 1.0, s);
}

}  // namespace snac
