// Outer residual for callers that cannot allocate device memory.
//
// Who needs this: some host programs own all device memory themselves -- a caching allocator, a
// fixed per-process memory budget, or a latency-sensitive loop in which the implicit device-wide
// synchronisation of cudaMalloc/cudaFree is not acceptable -- and so cannot create a plan (plan
// creation allocates its workspace). snac_residual_noalloc gives them the defect r = f - A p of a
// single block, the same result as snac_residual, with no plan and no allocation: its scratch (the
// block's cell widths, the 1-D operator coefficients and the per-CTA partial sums of the two norms)
// lives in one file-scope __device__ array of fixed size, which every GPU that loads this library
// holds until the process exits.
//
// The kernels below follow the plan path's coefficient rules and the residual kernel's chain of
// FMAs. The z end conditions are folded into the diagonal here (the plan keeps them as mirrored
// ghosts on the cell itself), and the norms are summed in a different grouping, so r and the norms
// match snac_residual to rounding, not bit for bit.
#include <cmath>

#include "kern_common.cuh"
#include "snac_impl.h"

namespace snac {
void set_error(const std::string& s);
}

namespace {
using namespace snac;

constexpr int NA_MAX_N = SNAC_NOALLOC_MAX_CELLS_PER_AXIS;
constexpr int NA_MAX_PART = 65536;          // per-CTA partial sums (grid is capped to fit)
constexpr int NA_ZSPLIT = 16;
// layout of the scratch, in doubles: widths [3][MAX_N] | coefficients [3][MAX_N] x {lo, hi, d, w} |
// partial sums [MAX_PART] x 4 | reduced sums [4]
constexpr size_t NA_W = 0;
constexpr size_t NA_C = NA_W + 3 * (size_t)NA_MAX_N;
constexpr size_t NA_P = NA_C + 3 * (size_t)NA_MAX_N * 4;
constexpr size_t NA_S = NA_P + (size_t)NA_MAX_PART * 4;
constexpr size_t NA_TOTAL = NA_S + 4;

static __device__ __align__(256) double g_noalloc_scratch[NA_TOTAL];

// Device address of the scratch in the current device's context. In host code the array's name
// only stands for the symbol; the address it has on the GPU comes from the runtime. It is looked up
// on every call (a host-side table lookup, small next to the launches): an address cached per device
// would go stale after cudaDeviceReset or any other change of the device's primary context.
int scratch_on_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return SNAC_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
  return SNAC_OK;
}

struct NaBlock {
  int n[3];
  int bc[3][2];
};

// 1-D operator pieces from the widths: the same rules and operation order as plan creation
// (x, y: coupling 1/(h w) with h = (w + w_nbr)/2, Dirichlet ghost -2/w^2; z: uniform dz).
__global__ void k_na_coefs(double* __restrict__ scr, NaBlock B) {
  const int a = blockIdx.y;
  const int n = B.n[a];
  const double* w = scr + NA_W + (size_t)a * NA_MAX_N;
  double* c = scr + NA_C + (size_t)a * NA_MAX_N * 4;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double lo = 0.0, hi = 0.0, d = 0.0;
    if (a < 2) {
      for (int sd = 0; sd < 2; ++sd) {
        const bool inner = sd == 0 ? i > 0 : i < n - 1;
        const int bc = B.bc[a][sd];
        double v = 0.0;
        if (inner || bc == SNAC_BC_PERIODIC) {
          const double wn = inner ? w[sd == 0 ? i - 1 : i + 1] : (sd == 0 ? w[n - 1] : w[0]);
          v = 1.0 / (0.5 * (w[i] + wn) * w[i]);
          d -= v;
        } else if (bc == SNAC_BC_DIRICHLET) {
          d -= 2.0 / (w[i] * w[i]);
        }
        (sd == 0 ? lo : hi) = v;
      }
    } else {
      const double iz2 = 1.0 / (w[0] * w[0]);
      const bool per = B.bc[2][0] == SNAC_BC_PERIODIC;
      lo = (i > 0 || per) ? iz2 : 0.0;
      hi = (i < n - 1 || per) ? iz2 : 0.0;
      d = -(lo + hi);
      if (!per && i == 0 && B.bc[2][0] == SNAC_BC_DIRICHLET) d -= 2.0 * iz2;
      if (!per && i == n - 1 && B.bc[2][1] == SNAC_BC_DIRICHLET) d -= 2.0 * iz2;
    }
    c[4 * i + 0] = lo;
    c[4 * i + 1] = hi;
    c[4 * i + 2] = d;
    c[4 * i + 3] = w[i];
  }
}

__device__ __forceinline__ void na_block_sum2(double& a, double& b, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    sh[warp] = a;
    sh[32 + warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    a = warp_sum(lane < nwarp ? sh[lane] : 0.0);
    b = warp_sum(lane < nwarp ? sh[32 + lane] : 0.0);
  }
}

// r = f - A p on one block; one partial {||r||^2, ||f||^2} per CTA (tiles of 32 x 8 cells,
// grid-stride over tiles, z planes strided by gridDim.y).
__global__ void __launch_bounds__(TILE_THREADS) k_na_resid(const double* __restrict__ scr_c, double* __restrict__ part,
                                                            NaBlock B, const double* __restrict__ f,
                                                            const double* __restrict__ p, double* __restrict__ r) {
  __shared__ double sh[64];
  const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
  const int ntx = (nx + TILE_X - 1) / TILE_X, nty = (ny + TILE_Y - 1) / TILE_Y;
  const double* cxa = scr_c;
  const double* cya = scr_c + (size_t)NA_MAX_N * 4;
  const double* cza = scr_c + (size_t)2 * NA_MAX_N * 4;
  const bool perx = B.bc[0][0] == SNAC_BC_PERIODIC, pery = B.bc[1][0] == SNAC_BC_PERIODIC;
  const bool perz = B.bc[2][0] == SNAC_BC_PERIODIC;
  const long long plane = (long long)nx * ny;
  double s_r = 0.0, s_f = 0.0;
  for (int t = blockIdx.x; t < ntx * nty; t += gridDim.x) {
    const int i = (t % ntx) * TILE_X + (threadIdx.x % TILE_X);
    const int j = (t / ntx) * TILE_Y + (threadIdx.x / TILE_X);
    if (i >= nx || j >= ny) continue;
    const double* cx = cxa + 4 * i;
    const double* cy = cya + 4 * j;
    const long long self = (long long)j * nx + i;
    const long long lw = i > 0 ? self - 1 : (perx ? self + nx - 1 : self);
    const long long le = i < nx - 1 ? self + 1 : (perx ? self - (nx - 1) : self);
    const long long ls = j > 0 ? self - nx : (pery ? self + (long long)(ny - 1) * nx : self);
    const long long ln = j < ny - 1 ? self + nx : (pery ? self - (long long)(ny - 1) * nx : self);
    const double dxy = cx[2] + cy[2];
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
      const double* cz = cza + 4 * k;
      const int kd = k > 0 ? k - 1 : (perz ? nz - 1 : k);
      const int ku = k < nz - 1 ? k + 1 : (perz ? 0 : k);
      const long long c = self + k * plane;
      const double pc = p[c];
      double ap = cx[0] * p[lw + k * plane];
      ap = fma(cx[1], p[le + k * plane], ap);
      ap = fma(cy[0], p[ls + k * plane], ap);
      ap = fma(cy[1], p[ln + k * plane], ap);
      ap = fma(cz[0], p[self + kd * plane], ap);
      ap = fma(cz[1], p[self + ku * plane], ap);
      ap = fma(dxy + cz[2], pc, ap);
      const double fv = f[c];
      const double rv = fv - ap;
      r[c] = rv;
      s_r = fma(rv, rv, s_r);
      s_f = fma(fv, fv, s_f);
    }
  }
  na_block_sum2(s_r, s_f, sh);
  if (threadIdx.x == 0) {
    double* o = part + 4 * ((long long)blockIdx.y * gridDim.x + blockIdx.x);
    o[0] = s_r;
    o[1] = s_f;
  }
}

__global__ void __launch_bounds__(1024) k_na_reduce(const double* __restrict__ part, int npart, double* __restrict__ sums) {
  __shared__ double sh[64];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < npart; i += blockDim.x) {
    a += part[4 * (long long)i];
    b += part[4 * (long long)i + 1];
  }
  na_block_sum2(a, b, sh);
  if (threadIdx.x == 0) {
    sums[0] = a;
    sums[1] = b;
  }
}

int fail(int code, const char* msg) {
  set_error(msg);
  return code;
}

}  // namespace

extern "C" int snac_residual_noalloc(const snac_block* block, const double* d_rhs, const double* d_p, double* d_r,
                                     double* h_norms, void* stream) {
  if (!block || !d_rhs || !d_p || !d_r || !h_norms) return fail(SNAC_ERR_INVALID_ARG, "NULL argument");
  NaBlock B{};
  for (int a = 0; a < 3; ++a) {
    const long long n = block->hi[a] - block->lo[a] + 1;
    if (n < 1) return fail(SNAC_ERR_INVALID_ARG, "bad lo/hi");
    if (n > NA_MAX_N)
      return fail(SNAC_ERR_INVALID_ARG,
                  "a block axis has more cells than the fixed scratch of snac_residual_noalloc holds (4096)");
    if (!block->h_dx[a]) return fail(SNAC_ERR_INVALID_ARG, "h_dx is NULL");
    B.n[a] = (int)n;
    for (int s = 0; s < 2; ++s) {
      const int bc = block->bc[a][s];
      if (bc != SNAC_BC_DIRICHLET && bc != SNAC_BC_NEUMANN && bc != SNAC_BC_PERIODIC)
        return fail(SNAC_ERR_INVALID_ARG, "snac_residual_noalloc takes one block: faces must be D, N or P");
      B.bc[a][s] = bc;
    }
    if ((B.bc[a][0] == SNAC_BC_PERIODIC) != (B.bc[a][1] == SNAC_BC_PERIODIC))
      return fail(SNAC_ERR_INVALID_ARG, "periodic needs both faces of the axis");
    for (int i = 0; i < B.n[a]; ++i)
      if (!(block->h_dx[a][i] > 0.0)) return fail(SNAC_ERR_INVALID_ARG, "cell widths must be > 0");
  }
  for (int k = 0; k < B.n[2]; ++k)
    if (std::fabs(block->h_dx[2][k] - block->h_dx[2][0]) > 1e-12 * block->h_dx[2][0])
      return fail(SNAC_ERR_LAYOUT, "the homogeneous direction must be uniform");
  double* scr = nullptr;
  int st = scratch_on_current_device(&scr);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < 3 && e == cudaSuccess; ++a)
    e = cudaMemcpyAsync(scr + NA_W + (size_t)a * NA_MAX_N, block->h_dx[a], B.n[a] * sizeof(double),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_na_coefs<<<dim3(16, 3), 256, 0, s>>>(scr, B);
    const int ntiles = ((B.n[0] + TILE_X - 1) / TILE_X) * ((B.n[1] + TILE_Y - 1) / TILE_Y);
    const int zs = B.n[2] < NA_ZSPLIT ? B.n[2] : NA_ZSPLIT;
    const int gx = ntiles < NA_MAX_PART / NA_ZSPLIT ? ntiles : NA_MAX_PART / NA_ZSPLIT;
    k_na_resid<<<dim3(gx, zs), TILE_THREADS, 0, s>>>(scr + NA_C, scr + NA_P, B, d_rhs, d_p, d_r);
    k_na_reduce<<<1, 1024, 0, s>>>(scr + NA_P, gx * zs, scr + NA_S);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_norms, scr + NA_S, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("snac_residual_noalloc: ") + cudaGetErrorString(e));
    return SNAC_ERR_CUDA;
  }
  return SNAC_OK;
}
