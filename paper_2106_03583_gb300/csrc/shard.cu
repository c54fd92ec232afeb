// The pencil stages of one rank in a solve sharded by wavenumber (App. A, Algorithm 3): transforms
// of the rank's columns, the outer FP64 residual of its pencil (with the neighbouring columns of
// other ranks supplied as halo columns), and the setup that lists those halo columns. The exchange
// of pencils and wavenumber slabs between ranks is the caller's (an all-to-all); the reduced
// equations of a slab are solved by snac_mode_solve on a wavenumber-range plan (solve.cu).
#include <algorithm>
#include <cstring>
#include <map>

#include "kern_common.cuh"
#include "snac_impl.h"

namespace snac {
void set_error(const std::string& s);
}

namespace {
using namespace snac;

constexpr int PEN_THREADS = 256;
constexpr int PEN_ZSPLIT = 16;
constexpr int PEN_SUMS = 5;

int cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return SNAC_ERR_CUDA;
}

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
  } while (0)

int check(snac_plan* P) {
  if (!P) return SNAC_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) {
    set_error("the current CUDA device is not the plan's device");
    return SNAC_ERR_INVALID_ARG;
  }
  return SNAC_OK;
}

template <int NV>
__device__ __forceinline__ void block_sum_n(double (&v)[NV], double* sh /* [NV][32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = warp_sum(v[k]);
    if (lane == 0) sh[k * 32 + warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(lane < nwarp ? sh[k * 32 + lane] : 0.0);
  }
}

// r = (f - fshift) - A p on a pencil (Eq. 8). One thread per pencil column, z planes strided by
// gridDim.y. cell[7 l ..]: block, i, j of column l and the p_ext columns of its W, E, S, N
// neighbours (the column itself on a physical face, where the coupling is zero). p_ext is
// [z][next]: the pencil's columns, then its halo columns. Partials per CTA (8 slots): ||r||^2,
// ||f - fshift||^2, sum V p, sum V (f - fshift), sum V |f - fshift|.
__global__ void __launch_bounds__(PEN_THREADS) k_pencil_resid(LevelView<double> L, const int* __restrict__ cell,
                                                               long long ncols, long long next,
                                                               const Coef<double>* __restrict__ cz, int nz,
                                                               int periodic_z, double zd, double dz,
                                                               const double* __restrict__ f,
                                                               const double* __restrict__ pe, double* __restrict__ r,
                                                               double fshift, double* __restrict__ part) {
  __shared__ double sh[PEN_SUMS * 32];
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[PEN_SUMS] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (l < ncols) {
    const int* c = cell + 7 * l;
    const BlockDev B = L.blk[c[0]];
    const Coef<double> cx = L.cx[B.xo + c[1]], cy = L.cy[B.yo + c[2]];
    const long long nw = c[3], ne = c[4], ns = c[5], nn = c[6];
    const double dg = cx.d + cy.d + zd;
    const double va = cx.w * cy.w * dz;
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
      const Coef<double> z = cz[k];
      const int kd = k > 0 ? k - 1 : (periodic_z ? nz - 1 : k);
      const int ku = k < nz - 1 ? k + 1 : (periodic_z ? 0 : k);
      const double* pk = pe + (long long)k * next;
      const double pc = pk[l];
      double ap = cx.lo * pk[nw];
      ap = fma(cx.hi, pk[ne], ap);
      ap = fma(cy.lo, pk[ns], ap);
      ap = fma(cy.hi, pk[nn], ap);
      ap = fma(z.lo, pe[(long long)kd * next + l], ap);
      ap = fma(z.hi, pe[(long long)ku * next + l], ap);
      ap = fma(dg, pc, ap);
      const double fv = f[(long long)k * ncols + l] - fshift;
      const double rv = fv - ap;
      r[(long long)k * ncols + l] = rv;
      acc[0] = fma(rv, rv, acc[0]);
      acc[1] = fma(fv, fv, acc[1]);
      acc[2] = fma(va, pc, acc[2]);
      acc[3] = fma(va, fv, acc[3]);
      acc[4] = fma(va, fabs(fv), acc[4]);
    }
  }
  block_sum_n<PEN_SUMS>(acc, sh);
  if (threadIdx.x == 0) {
    double* o = part + 8 * ((long long)blockIdx.y * gridDim.x + blockIdx.x);
    for (int k = 0; k < PEN_SUMS; ++k) o[k] = acc[k];
  }
}

// Fixed-order sum of the partials (one CTA).
__global__ void __launch_bounds__(1024) k_pencil_reduce(const double* __restrict__ part, int npart,
                                                        double* __restrict__ out) {
  __shared__ double sh[PEN_SUMS * 32];
  double acc[PEN_SUMS] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < npart; i += blockDim.x)
    for (int k = 0; k < PEN_SUMS; ++k) acc[k] += part[8 * (long long)i + k];
  block_sum_n<PEN_SUMS>(acc, sh);
  if (threadIdx.x == 0)
    for (int k = 0; k < PEN_SUMS; ++k) out[k] = acc[k];
}

// The four x-y neighbours of cell (i, j) of block b as level-0 plane cells (host; the same face
// rules as the kernels: the adjacent cell, the facing cell of a connected or periodic block, or the
// cell itself on a physical face).
void plane_neighbours(const std::vector<BlockDev>& blk, int b, int i, int j, long long (&nb)[4]) {
  const BlockDev& B = blk[b];
  const long long self = B.off + (long long)j * B.nx + i;
  for (long long& v : nb) v = self;
  if (i > 0) nb[0] = self - 1;
  else if (B.nbr[0] >= 0) nb[0] = blk[B.nbr[0]].off + (long long)j * blk[B.nbr[0]].nx + (blk[B.nbr[0]].nx - 1);
  if (i < B.nx - 1) nb[1] = self + 1;
  else if (B.nbr[1] >= 0) nb[1] = blk[B.nbr[1]].off + (long long)j * blk[B.nbr[1]].nx;
  if (j > 0) nb[2] = self - B.nx;
  else if (B.nbr[2] >= 0) nb[2] = blk[B.nbr[2]].off + (long long)(blk[B.nbr[2]].ny - 1) * blk[B.nbr[2]].nx + i;
  if (j < B.ny - 1) nb[3] = self + B.nx;
  else if (B.nbr[3] >= 0) nb[3] = blk[B.nbr[3]].off + i;
}

}  // namespace

extern "C" {

int snac_pencil_forward(snac_plan* plan, int64_t ncols, const double* d_in, void* d_modes, void* stream) {
  int st = check(plan);
  if (st) return st;
  if (!d_in || !d_modes || ncols < 1) return SNAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_pencil_forward(plan, ncols, d_in, d_modes, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(plan);
  return SNAC_OK;
}

int snac_pencil_backward_update(snac_plan* plan, int64_t ncols, const void* d_modes, double* d_p, void* stream) {
  int st = check(plan);
  if (st) return st;
  if (!d_modes || !d_p || ncols < 1) return SNAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_pencil_backward(plan, ncols, d_modes, d_p, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(plan);
  return SNAC_OK;
}

int snac_pencil_setup(snac_plan* plan, int64_t c0, int64_t ncols, int64_t* h_halo, int64_t max_halo, int64_t* nhalo) {
  int st = check(plan);
  if (st) return st;
  const HostLevel& l0 = plan->lev[0];
  if (!nhalo || (max_halo > 0 && !h_halo) || c0 < 0 || ncols < 1 || c0 + ncols > l0.ncell || ncols >= (1LL << 30))
    return SNAC_ERR_INVALID_ARG;
  // block, i, j and plane neighbours of every pencil cell; the halo: neighbours outside the pencil
  std::vector<int> cell(7 * (size_t)ncols);
  std::vector<long long> nbp(4 * (size_t)ncols);
  std::vector<long long> halo;
  int b = 0;
  for (long long l = 0; l < ncols; ++l) {
    const long long c = c0 + l;
    while (b + 1 < l0.nblk && l0.blk[b + 1].off <= c) ++b;
    const BlockDev& B = l0.blk[b];
    const int i = (int)((c - B.off) % B.nx), j = (int)((c - B.off) / B.nx);
    long long nb[4];
    plane_neighbours(l0.blk, b, i, j, nb);
    cell[7 * l] = b;
    cell[7 * l + 1] = i;
    cell[7 * l + 2] = j;
    for (int f = 0; f < 4; ++f) {
      nbp[4 * l + f] = nb[f];
      if (nb[f] < c0 || nb[f] >= c0 + ncols) halo.push_back(nb[f]);
    }
  }
  std::sort(halo.begin(), halo.end());
  halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
  *nhalo = (int64_t)halo.size();
  if ((int64_t)halo.size() > max_halo) {
    set_error("the pencil's halo has more columns than max_halo");
    return SNAC_ERR_INVALID_ARG;
  }
  for (long long l = 0; l < ncols; ++l)
    for (int f = 0; f < 4; ++f) {
      const long long v = nbp[4 * l + f];
      long long col;
      if (v >= c0 && v < c0 + ncols) col = v - c0;
      else col = ncols + (std::lower_bound(halo.begin(), halo.end(), v) - halo.begin());
      cell[7 * l + 3 + f] = (int)col;
    }
  std::copy(halo.begin(), halo.end(), h_halo);
  for (void* p : plan->pen_allocs) cudaFree(p);
  plan->pen_allocs.clear();
  plan->pen_ncols = 0;
  const int gx = (int)((ncols + PEN_THREADS - 1) / PEN_THREADS), gy = std::min(plan->nzt, PEN_ZSPLIT);
  plan->pen_nparts = gx * gy;
  CK(cudaMalloc((void**)&plan->d_pen_cell, cell.size() * sizeof(int)));
  plan->pen_allocs.push_back(plan->d_pen_cell);
  CK(cudaMalloc((void**)&plan->d_pen_part, (size_t)plan->pen_nparts * 8 * sizeof(double)));
  plan->pen_allocs.push_back(plan->d_pen_part);
  CK(cudaMemcpy(plan->d_pen_cell, cell.data(), cell.size() * sizeof(int), cudaMemcpyHostToDevice));
  plan->pen_c0 = c0;
  plan->pen_ncols = ncols;
  plan->pen_nhalo = (long long)halo.size();
  return SNAC_OK;
}

int snac_pencil_residual(snac_plan* plan, const double* d_f, const double* d_p_ext, double* d_r, double fshift,
                         double* h_sums, void* stream) {
  int st = check(plan);
  if (st) return st;
  if (!d_f || !d_p_ext || !d_r || !h_sums || plan->pen_ncols < 1) return SNAC_ERR_INVALID_ARG;
  snac_plan* P = plan;
  cudaStream_t s = (cudaStream_t)stream;
  const long long ncols = P->pen_ncols;
  const dim3 grid((unsigned)((ncols + PEN_THREADS - 1) / PEN_THREADS), (unsigned)std::min(P->nzt, PEN_ZSPLIT));
  const double n3 = (double)ncols * P->nzt;
  {
    LaunchScope ls(P, K_FIELD3D, 24.0 * n3, 23.0 * n3, s);
    k_pencil_resid<<<grid, PEN_THREADS, 0, s>>>(level_view<double>(P->lev[0]), P->d_pen_cell, ncols,
                                                ncols + P->pen_nhalo, P->d_cz, P->nzt, P->kind == KIND_PP, P->cz[0].d,
                                                P->dz, d_f, d_p_ext, d_r, fshift, P->d_pen_part);
  }
  CK(cudaGetLastError());
  {
    LaunchScope ls(P, K_REDUCE, 64.0 * P->pen_nparts, 5.0 * P->pen_nparts, s);
    k_pencil_reduce<<<1, 1024, 0, s>>>(P->d_pen_part, P->pen_nparts, P->d_sums);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h_sums, P->d_sums, PEN_SUMS * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(P);
  return SNAC_OK;
}

}  // extern "C"
