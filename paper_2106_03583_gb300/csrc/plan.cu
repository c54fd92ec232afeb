// Plan creation: validation of the block graph, multigrid hierarchy, operator coefficients,
// eigenvalue shifts, transform twiddles, coarsest-level factorisation and device workspace.
//
// Discretisation (Eq. 8, Sec. 2; general non-uniform form, footnote of Sec. 3.3): cell-centred
// pressure, row of cell i along a stretched axis
//     [(p_{i+1} - p_i)/h_{i+1/2} - (p_i - p_{i-1})/h_{i-1/2}] / w_i,   h = (w_i + w_nbr)/2,
// homogeneous Dirichlet / Neumann faces by a mirrored ghost (-p / +p at distance w_i), block-block
// and periodic faces by the connected cell (Sec. 3.1). The homogeneous axis z is uniform and
// diagonalised by the transform of Table 1 with eigenvalues lambda_q = 2 (cos(kappa_q dz) - 1).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "fused_tab.h"
#include "kern_common.cuh"
#include "snac_impl.h"

using namespace snac;

namespace snac {
thread_local std::string g_last_error;
void set_error(const std::string& s) { g_last_error = s; }
}  // namespace snac

namespace {

struct HBlock {
  long long lo[3], hi[3];
  int n[3];
  std::vector<double> w[3];
  int bc[3][2];
  int nbr[3][2];
};

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

// Face number of (axis, side): W, E, S, N = 0..3.
inline int face(int axis, int side) { return 2 * axis + side; }

int validate(int nb, const snac_block* in, std::vector<HBlock>& out) {
  out.resize(nb);
  for (int b = 0; b < nb; ++b) {
    const snac_block& s = in[b];
    HBlock& h = out[b];
    for (int a = 0; a < 3; ++a) {
      h.lo[a] = s.lo[a];
      h.hi[a] = s.hi[a];
      long long n = s.hi[a] - s.lo[a] + 1;
      if (n < 1 || n > (1LL << 24)) return fail(SNAC_ERR_INVALID_ARG, "block " + std::to_string(b) + ": bad lo/hi");
      h.n[a] = (int)n;
      if (!s.h_dx[a]) return fail(SNAC_ERR_INVALID_ARG, "block " + std::to_string(b) + ": h_dx is NULL");
      h.w[a].assign(s.h_dx[a], s.h_dx[a] + n);
      for (double w : h.w[a])
        if (!(w > 0.0) || !std::isfinite(w))
          return fail(SNAC_ERR_INVALID_ARG, "block " + std::to_string(b) + ": cell widths must be finite and > 0");
      for (int sd = 0; sd < 2; ++sd) {
        h.bc[a][sd] = s.bc[a][sd];
        h.nbr[a][sd] = s.nbr[a][sd];
        if (h.bc[a][sd] < SNAC_BC_DIRICHLET || h.bc[a][sd] > SNAC_BC_BLOCK)
          return fail(SNAC_ERR_INVALID_ARG, "block " + std::to_string(b) + ": unknown face kind");
      }
    }
  }
  // homogeneous axis: same n_z, the same uniform widths, the same pair, not split into blocks
  const HBlock& b0 = out[0];
  const int nz = b0.n[2];
  for (int b = 0; b < nb; ++b) {
    const HBlock& h = out[b];
    if (h.n[2] != nz) return fail(SNAC_ERR_LAYOUT, "all blocks must have the same n_z");
    for (int sd = 0; sd < 2; ++sd)
      if (h.bc[2][sd] != b0.bc[2][sd]) return fail(SNAC_ERR_LAYOUT, "all blocks must share the z boundary pair");
    for (int k = 0; k < nz; ++k)
      if (h.w[2][k] != b0.w[2][k]) return fail(SNAC_ERR_LAYOUT, "all blocks must share the z grid");
  }
  for (int k = 0; k < nz; ++k)
    if (std::fabs(b0.w[2][k] - b0.w[2][0]) > 1e-12 * b0.w[2][0])
      return fail(SNAC_ERR_LAYOUT, "the homogeneous direction must be uniform (Sec. 2)");
  if (b0.bc[2][0] == SNAC_BC_BLOCK || b0.bc[2][1] == SNAC_BC_BLOCK)
    return fail(SNAC_ERR_LAYOUT, "blocks cannot be connected along the homogeneous direction");
  if ((b0.bc[2][0] == SNAC_BC_PERIODIC) != (b0.bc[2][1] == SNAC_BC_PERIODIC))
    return fail(SNAC_ERR_LAYOUT, "a periodic z needs both z faces periodic");
  if (nz % 2) return fail(SNAC_ERR_LAYOUT, "n_z must be even (Table 1)");
  if (nz > MAX_NZ) return fail(SNAC_ERR_LAYOUT, "n_z above the supported maximum 4096");
  // x-y connectivity
  for (int b = 0; b < nb; ++b) {
    const HBlock& h = out[b];
    for (int a = 0; a < 2; ++a) {
      const int o = 1 - a;
      if ((h.bc[a][0] == SNAC_BC_PERIODIC) != (h.bc[a][1] == SNAC_BC_PERIODIC))
        return fail(SNAC_ERR_LAYOUT, "block " + std::to_string(b) + ": periodic needs both faces of the axis");
      for (int sd = 0; sd < 2; ++sd) {
        if (h.bc[a][sd] != SNAC_BC_BLOCK) continue;
        const int c = h.nbr[a][sd];
        if (c < 0 || c >= nb) return fail(SNAC_ERR_LAYOUT, "block " + std::to_string(b) + ": bad neighbour id");
        const HBlock& g = out[c];
        if (g.bc[a][1 - sd] != SNAC_BC_BLOCK || g.nbr[a][1 - sd] != b)
          return fail(SNAC_ERR_LAYOUT, "block " + std::to_string(b) + ": connectivity with block " +
                                           std::to_string(c) + " is not symmetric");
        if (g.lo[o] != h.lo[o] || g.hi[o] != h.hi[o])
          return fail(SNAC_ERR_LAYOUT, "block " + std::to_string(b) + ": face shared with block " +
                                           std::to_string(c) + " does not coincide");
        if (g.w[o] != h.w[o])
          return fail(SNAC_ERR_LAYOUT, "block " + std::to_string(b) + ": grid not congruent with block " +
                                           std::to_string(c) + " (Sec. 3.1)");
      }
    }
  }
  return SNAC_OK;
}

// Cyclic Jacobi eigenvalue iteration for a small symmetric matrix S (n x n, row-major).
// On return S is (numerically) diagonal with the eigenvalues, Q holds the eigenvectors as columns.
void jacobi_eigen(int n, std::vector<double>& S, std::vector<double>& Q) {
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  double norm = 0.0;
  for (double v : S) norm += v * v;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += S[(size_t)p * n + q] * S[(size_t)p * n + q];
    if (off <= 1e-32 * norm) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = S[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = S[(size_t)p * n + p], aqq = S[(size_t)q * n + q];
        const double th = (aqq - app) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double skp = S[(size_t)k * n + p], skq = S[(size_t)k * n + q];
          S[(size_t)k * n + p] = c * skp - s * skq;
          S[(size_t)k * n + q] = s * skp + c * skq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double spk = S[(size_t)p * n + k], sqk = S[(size_t)q * n + k];
          S[(size_t)p * n + k] = c * spk - s * sqk;
          S[(size_t)q * n + k] = s * spk + c * sqk;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
          Q[(size_t)k * n + p] = c * qkp - s * qkq;
          Q[(size_t)k * n + q] = s * qkp + c * qkq;
        }
      }
    }
  }
}

template <typename T>
int dmalloc(snac_plan* P, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? SNAC_ERR_OOM : SNAC_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  P->allocs.push_back(p);
  P->bytes += count * sizeof(T);
  *ptr = (T*)p;
  return SNAC_OK;
}

template <typename T>
int upload(snac_plan* P, T** ptr, const std::vector<T>& v) {
  int st = dmalloc(P, ptr, v.size());
  if (st) return st;
  if (!v.empty() && cudaMemcpy(*ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(SNAC_ERR_CUDA, "cudaMemcpy upload failed");
  return SNAC_OK;
}

template <typename T>
std::vector<Coef<float>> to32(const std::vector<Coef<T>>& v) {
  std::vector<Coef<float>> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = {(float)v[i].lo, (float)v[i].hi, (float)v[i].d, (float)v[i].w};
  return o;
}
std::vector<PW<float>> to32(const std::vector<PW<double>>& v) {
  std::vector<PW<float>> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = {(float)v[i].self, (float)v[i].nbr};
  return o;
}
std::vector<float> to32(const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); }

// Widths of every block along one axis at a level (level-0 widths summed in groups of 2^l).
std::vector<double> level_widths(const std::vector<double>& w0, int l) {
  const int g = 1 << l;
  std::vector<double> w(w0.size() / g, 0.0);
  for (size_t i = 0; i < w.size(); ++i)
    for (int k = 0; k < g; ++k) w[i] += w0[i * g + k];
  return w;
}

// 1-D operator pieces along one axis of one block: coupling to the lower/upper neighbour with the
// centre distance h = (w + w_nbr)/2, or the ghost rule of a physical face.
void axis_coefs(const std::vector<double>& w, int bc_lo, int bc_hi, double w_nlo, double w_nhi,
                std::vector<Coef<double>>& out) {
  const int n = (int)w.size();
  for (int i = 0; i < n; ++i) {
    Coef<double> c{0.0, 0.0, 0.0, w[i]};
    for (int sd = 0; sd < 2; ++sd) {
      const bool inner = sd == 0 ? i > 0 : i < n - 1;
      const int bc = sd == 0 ? bc_lo : bc_hi;
      double a = 0.0;
      if (inner || bc == SNAC_BC_BLOCK || bc == SNAC_BC_PERIODIC) {
        const double wn = inner ? w[sd == 0 ? i - 1 : i + 1] : (sd == 0 ? w_nlo : w_nhi);
        a = 1.0 / (0.5 * (w[i] + wn) * w[i]);
        c.d -= a;
      } else if (bc == SNAC_BC_DIRICHLET) {
        c.d -= 2.0 / (w[i] * w[i]);
      }
      (sd == 0 ? c.lo : c.hi) = a;
    }
    out.push_back(c);
  }
}

int build_levels(snac_plan* P, const std::vector<HBlock>& hb) {
  const int nb = (int)hb.size();
  long long lox = hb[0].lo[0], loy = hb[0].lo[1];
  for (const HBlock& h : hb) {
    lox = std::min(lox, h.lo[0]);
    loy = std::min(loy, h.lo[1]);
  }
  // number of levels
  int L = 0;
  for (;;) {
    long long ncell = 0;
    bool ok = true;
    for (const HBlock& h : hb) {
      const int nx = h.n[0] >> L, ny = h.n[1] >> L;
      ncell += (long long)nx * ny;
      const long long rx = h.lo[0] - lox, ry = h.lo[1] - loy;
      if (nx % 2 || ny % 2 || nx < 4 || ny < 4) ok = false;
      if (rx % (2LL << L) || ry % (2LL << L)) ok = false;
    }
    if (ncell <= P->max_coarse || !ok) break;
    ++L;
  }
  P->lev.assign(L + 1, HostLevel());
  for (int l = 0; l <= L; ++l) {
    HostLevel& lv = P->lev[l];
    lv.nblk = nb;
    std::vector<std::vector<double>> wx(nb), wy(nb);
    for (int b = 0; b < nb; ++b) {
      wx[b] = level_widths(hb[b].w[0], l);
      wy[b] = level_widths(hb[b].w[1], l);
    }
    long long off = 0;
    int xo = 0, yo = 0;
    for (int b = 0; b < nb; ++b) {
      BlockDev d{};
      d.off = off;
      d.nx = (int)wx[b].size();
      d.ny = (int)wy[b].size();
      d.xo = xo;
      d.yo = yo;
      for (int a = 0; a < 2; ++a)
        for (int sd = 0; sd < 2; ++sd) {
          const int bc = hb[b].bc[a][sd];
          d.nbr[face(a, sd)] = bc == SNAC_BC_BLOCK ? hb[b].nbr[a][sd] : (bc == SNAC_BC_PERIODIC ? b : -1);
        }
      const long long rx = (hb[b].lo[0] - lox) >> l, ry = (hb[b].lo[1] - loy) >> l;
      d.par = (int)((rx + ry) & 1);
      lv.blk.push_back(d);
      off += (long long)d.nx * d.ny;
      xo += d.nx;
      yo += d.ny;
      for (int y0 = 0; y0 < d.ny; y0 += TILE_Y)
        for (int x0 = 0; x0 < d.nx; x0 += TILE_X) lv.tiles.push_back({b, x0, y0, 0});
    }
    lv.ncell = off;
    for (int b = 0; b < nb; ++b) {
      const BlockDev& d = lv.blk[b];
      auto nbw = [&](int a, int sd) -> double {  // width of the connected cell across a face
        const int c = d.nbr[face(a, sd)];
        if (c < 0) return 0.0;
        const std::vector<double>& w = a == 0 ? wx[c] : wy[c];
        return sd == 0 ? w.back() : w.front();
      };
      axis_coefs(wx[b], hb[b].bc[0][0], hb[b].bc[0][1], nbw(0, 0), nbw(0, 1), lv.cx);
      axis_coefs(wy[b], hb[b].bc[1][0], hb[b].bc[1][1], nbw(1, 0), nbw(1, 1), lv.cy);
    }
  }
  // transfer weights between level l (fine) and l+1 (coarse)
  for (int l = 0; l < L; ++l) {
    HostLevel& fl = P->lev[l];
    const HostLevel& cl = P->lev[l + 1];
    for (int b = 0; b < nb; ++b) {
      for (int a = 0; a < 2; ++a) {
        const BlockDev& fd = fl.blk[b];
        const BlockDev& cd = cl.blk[b];
        const int n = a == 0 ? fd.nx : fd.ny;
        const int nco = a == 0 ? cd.nx : cd.ny;
        const Coef<double>* fc = (a == 0 ? fl.cx.data() + fd.xo : fl.cy.data() + fd.yo);
        const Coef<double>* cc = (a == 0 ? cl.cx.data() + cd.xo : cl.cy.data() + cd.yo);
        for (int i = 0; i < n; ++i) {
          const int I = i / 2, sd = i & 1;
          // fine centre to parent centre: half the sibling's width
          const double dist = 0.5 * fc[i ^ 1].w;
          const double W = cc[I].w;
          double self = 0.0, nbrw = 0.0;
          const bool inner = sd == 0 ? I > 0 : I < nco - 1;
          const int bc = hb[b].bc[a][sd];
          if (inner || bc == SNAC_BC_BLOCK || bc == SNAC_BC_PERIODIC) {
            double Wn;
            if (inner) {
              Wn = cc[sd == 0 ? I - 1 : I + 1].w;
            } else {
              const int c = cd.nbr[face(a, sd)];
              const BlockDev& nd = cl.blk[c];
              const Coef<double>* nc = a == 0 ? cl.cx.data() + nd.xo : cl.cy.data() + nd.yo;
              const int nn = a == 0 ? nd.nx : nd.ny;
              Wn = sd == 0 ? nc[nn - 1].w : nc[0].w;
            }
            const double wgt = dist / (0.5 * (W + Wn));
            self = -wgt;
            nbrw = wgt;
          } else if (bc == SNAC_BC_DIRICHLET) {
            self = -2.0 * dist / W;  // ghost -e_C at the mirrored centre, distance W
          }
          (a == 0 ? fl.px : fl.py).push_back({self, nbrw});
          (a == 0 ? fl.rx : fl.ry).push_back(fc[i].w / W);
        }
      }
    }
  }
  return SNAC_OK;
}

double mode_lambda(int kind, int n, int q) {
  double m;
  switch (kind) {
    case KIND_PP: m = q; break;
    case KIND_NN: m = 0.5 * q; break;
    case KIND_DD: m = 0.5 * (q + 1); break;
    default: m = 0.25 * (2 * q + 1); break;
  }
  return 2.0 * (std::cos(2.0 * M_PI * m / n) - 1.0);
}

// Weight w_q with sum_k x_k^2 = sum_q w_q Xhat_q^2 for the unnormalised transforms of Table 1.
double parseval_weight(int kind, int n, int q) {
  switch (kind) {
    case KIND_PP: return (q == 0 || q == n / 2) ? 1.0 / n : 2.0 / n;
    case KIND_NN: return q == 0 ? 0.25 / n : 0.5 / n;
    case KIND_DD: return q == n - 1 ? 0.25 / n : 0.5 / n;
    default: return 0.5 / n;
  }
}

int build_coarse(snac_plan* P) {
  const HostLevel& lv = P->lev.back();
  const int n = (int)lv.ncell;
  if (n > MAX_COARSE)
    return fail(SNAC_ERR_LAYOUT, "the coarsest multigrid plane has " + std::to_string(n) +
                                     " cells (> 256): blocks must be divisible by 2 more often");
  P->nc = n;
  std::vector<double> A((size_t)n * n, 0.0), area(n);
  for (int b = 0; b < lv.nblk; ++b) {
    const BlockDev& d = lv.blk[b];
    for (int j = 0; j < d.ny; ++j)
      for (int i = 0; i < d.nx; ++i) {
        const Coef<double>& cx = lv.cx[d.xo + i];
        const Coef<double>& cy = lv.cy[d.yo + j];
        const long long row = d.off + (long long)j * d.nx + i;
        area[row] = cx.w * cy.w;
        A[row * n + row] += cx.d + cy.d;
        auto cell = [&](int bb, int ii, int jj) { return lv.blk[bb].off + (long long)jj * lv.blk[bb].nx + ii; };
        if (cx.lo != 0.0) {
          const long long c = i > 0 ? cell(b, i - 1, j) : cell(d.nbr[0], lv.blk[d.nbr[0]].nx - 1, j);
          A[row * n + c] += cx.lo;
        }
        if (cx.hi != 0.0) {
          const long long c = i < d.nx - 1 ? cell(b, i + 1, j) : cell(d.nbr[1], 0, j);
          A[row * n + c] += cx.hi;
        }
        if (cy.lo != 0.0) {
          const long long c = j > 0 ? cell(b, i, j - 1) : cell(d.nbr[2], i, lv.blk[d.nbr[2]].ny - 1);
          A[row * n + c] += cy.lo;
        }
        if (cy.hi != 0.0) {
          const long long c = j < d.ny - 1 ? cell(b, i, j + 1) : cell(d.nbr[3], i, 0);
          A[row * n + c] += cy.hi;
        }
      }
  }
  // S = V^1/2 A V^-1/2 is symmetric because V A is (finite-volume fluxes)
  std::vector<double> S((size_t)n * n), sqa(n);
  for (int i = 0; i < n; ++i) sqa[i] = std::sqrt(area[i]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) S[(size_t)i * n + j] = sqa[i] * A[(size_t)i * n + j] / sqa[j];
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double m = 0.5 * (S[(size_t)i * n + j] + S[(size_t)j * n + i]);
      S[(size_t)i * n + j] = S[(size_t)j * n + i] = m;
    }
  std::vector<double> Q;
  jacobi_eigen(n, S, Q);
  std::vector<double> lam(n);
  for (int i = 0; i < n; ++i) lam[i] = S[(size_t)i * n + i];
  P->null_index = -1;
  if (P->singular) {
    int k = 0;
    for (int i = 1; i < n; ++i)
      if (std::fabs(lam[i]) < std::fabs(lam[k])) k = i;
    P->null_index = k;
  }
  std::vector<double> QT((size_t)n * n);  // its transpose, so that both products of the solve read whole rows
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) QT[(size_t)k * n + i] = Q[(size_t)i * n + k];
  int st;
  if ((st = upload(P, &P->d_Q, Q)) || (st = upload(P, &P->d_QT, QT)) || (st = upload(P, &P->d_lam, lam)) ||
      (st = upload(P, &P->d_sqa, sqa)))
    return st;
  return SNAC_OK;
}

int build_twiddles(snac_plan* P) {
  const int n = P->nzt, m = n / 2;
  TwiddleOffsets& t = P->tw;
  t.fft = 0;
  t.twn = t.fft + m;
  t.tw2n = t.twn + m + 1;
  t.tw4a = t.tw2n + n + 1;
  t.tw4b = t.tw4a + m;
  t.total = t.tw4b + m;
  std::vector<double> tw(2 * (size_t)t.total);
  auto put = [&](int idx, double ang) {
    tw[2 * idx] = std::cos(ang);
    tw[2 * idx + 1] = std::sin(ang);
  };
  for (int k = 0; k < m; ++k) put(t.fft + k, -2.0 * M_PI * k / m);
  for (int k = 0; k <= m; ++k) put(t.twn + k, -2.0 * M_PI * k / n);
  for (int k = 0; k <= n; ++k) put(t.tw2n + k, -M_PI * k / (2.0 * n));
  for (int k = 0; k < m; ++k) put(t.tw4a + k, -M_PI * (4.0 * k + 1.0) / (4.0 * n));
  for (int k = 0; k < m; ++k) put(t.tw4b + k, -M_PI * k / (double)n);
  int st;
  if ((st = upload(P, &P->d_tw64, tw))) return st;
  if ((st = upload(P, &P->d_tw32, to32(tw)))) return st;
  return SNAC_OK;
}

int build_chunks(snac_plan* P, int tc, std::vector<ChunkDev>& ch, ChunkDev** d) {
  const HostLevel& l0 = P->lev[0];
  for (int b = 0; b < l0.nblk; ++b) {
    const int cells = l0.blk[b].nx * l0.blk[b].ny;
    for (int c0 = 0; c0 < cells; c0 += tc) ch.push_back({b, c0, std::min(tc, cells - c0), 0});
  }
  return upload(P, d, ch);
}

int upload_level(snac_plan* P, HostLevel& lv, size_t inner) {
  int st;
  if ((st = upload(P, &lv.d_blk, lv.blk)) || (st = upload(P, &lv.d_tiles, lv.tiles)) ||
      (st = upload(P, &lv.d_cx64, lv.cx)) || (st = upload(P, &lv.d_cy64, lv.cy)) ||
      (st = upload(P, &lv.d_cx32, to32(lv.cx))) || (st = upload(P, &lv.d_cy32, to32(lv.cy))))
    return st;
  {
    // cx.d + cy.d per plane cell: the residual kernels add only the mode's shift (same rounding as
    // forming the three-term sum in that order)
    std::vector<double> dxy(lv.ncell);
    for (const BlockDev& d : lv.blk)
      for (int j = 0; j < d.ny; ++j)
        for (int i = 0; i < d.nx; ++i) dxy[d.off + (long long)j * d.nx + i] = lv.cx[d.xo + i].d + lv.cy[d.yo + j].d;
    if ((st = upload(P, &lv.d_dxy64, dxy)) || (st = upload(P, &lv.d_dxy32, to32(dxy)))) return st;
  }
  if (!lv.px.empty()) {
    // the device copy of the x weights carries the parent's unit weight: self_x + 1, so that the
    // prolongation forms the parent's total weight (1 + self_x) + self_y with one addition
    std::vector<PW<double>> px1 = lv.px;
    for (PW<double>& w : px1) w.self += 1.0;
    // per plane cell: the restriction weight rx * ry and the parent's prolongation weight
    // (1 + self_x) + self_y, as the kernels would form them (one FP64 operation fewer per use)
    std::vector<double> wr(lv.ncell), wp(lv.ncell);
    for (const BlockDev& d : lv.blk)
      for (int j = 0; j < d.ny; ++j)
        for (int i = 0; i < d.nx; ++i) {
          const long long c = d.off + (long long)j * d.nx + i;
          wr[c] = lv.rx[d.xo + i] * lv.ry[d.yo + j];
          wp[c] = px1[d.xo + i].self + lv.py[d.yo + j].self;
        }
    if ((st = upload(P, &lv.d_wr64, wr)) || (st = upload(P, &lv.d_wr32, to32(wr))) ||
        (st = upload(P, &lv.d_wp64, wp)) || (st = upload(P, &lv.d_wp32, to32(wp))) ||
        (st = upload(P, &lv.d_px64, px1)) || (st = upload(P, &lv.d_py64, lv.py)) ||
        (st = upload(P, &lv.d_px32, to32(px1))) || (st = upload(P, &lv.d_py32, to32(lv.py))) ||
        (st = upload(P, &lv.d_rx64, lv.rx)) || (st = upload(P, &lv.d_ry64, lv.ry)) ||
        (st = upload(P, &lv.d_rx32, to32(lv.rx))) || (st = upload(P, &lv.d_ry32, to32(lv.ry))))
      return st;
  }
  char* u = nullptr;
  char* f = nullptr;
  const size_t cnt = (size_t)P->nz * lv.ncell * inner;
  if ((st = dmalloc(P, &u, cnt)) || (st = dmalloc(P, &f, cnt))) return st;
  lv.d_u = u;
  lv.d_f = f;
  return SNAC_OK;
}

void free_plan(snac_plan* P) {
  if (!P) return;
  profile_release(P);
  for (auto& kv : P->round_graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (P->capture_stream) cudaStreamDestroy(P->capture_stream);
  for (void* p : P->allocs) cudaFree(p);
  for (void* p : P->pen_tallocs) cudaFree(p);
  for (void* p : P->pen_allocs) cudaFree(p);
  if (P->h_sums) cudaFreeHost(P->h_sums);
  if (P->h_mode_norm2) cudaFreeHost(P->h_mode_norm2);
  if (P->h_active) cudaFreeHost(P->h_active);
  if (P->h_check) cudaFreeHost(P->h_check);
  if (P->h_cycles) cudaFreeHost(P->h_cycles);
  if (P->h_wait) cudaFreeHost(P->h_wait);
  delete P;
}

// Per-tile tables of the fused kernels of one level (the window's region blocks, coefficients,
// weights and plane offsets, in the shared-memory layout of FusedTab).
template <typename T>
int upload_fused_tabs(snac_plan* P, HostLevel& lv, const HostLevel& lc) {
  auto region = [](int i, int n) { return i < 0 ? 0 : (i >= n ? 2 : 1); };
  auto local = [](int i, int r, int n, int nr) { return r == 0 ? i + nr : (r == 2 ? i - n : i); };
  auto nb = [&](int b, int f) { return b < 0 ? -1 : lv.blk[b].nbr[f]; };
  if (lv.ncell >= (1LL << 30) || lc.ncell >= (1LL << 30))
    return fail(SNAC_ERR_INVALID_ARG, "fused levels need planes of fewer than 2^30 cells (set fused = 0)");
  std::vector<FusedTab<T>> tabs(lv.ftiles.size());
  const int H = FUSED_HALO;
  for (size_t n = 0; n < lv.ftiles.size(); ++n) {
    const TileDev& t = lv.ftiles[n];
    FusedTab<T>& tb = tabs[n];
    std::memset(&tb, 0, sizeof tb);
    const BlockDev& d = lv.blk[t.b];
    const BlockDev& dc = lc.blk[t.b];
    // the blocks around the tile's block, [ry][rx]: faces directly, corners through either neighbour
    const int W = d.nbr[0], E = d.nbr[1], S = d.nbr[2], N = d.nbr[3];
    const int R[3][3] = {{nb(W, 2) >= 0 ? nb(W, 2) : nb(S, 0), S, nb(E, 2) >= 0 ? nb(E, 2) : nb(S, 1)},
                         {W, t.b, E},
                         {nb(W, 3) >= 0 ? nb(W, 3) : nb(N, 0), N, nb(E, 3) >= 0 ? nb(E, 3) : nb(N, 1)}};
    tb.tw = std::min(FTILE_X, d.nx - t.x0);
    tb.th = std::min(FTILE_Y, d.ny - t.y0);
    const int x0w = t.x0 - H, y0w = t.y0 - H;  // even
    tb.pbase = ((d.par + x0w + y0w) % 2 + 2) % 2;
    tb.cnx = dc.nx;
    tb.cout0 = (int)(dc.off + (long long)(y0w / 2) * dc.nx + x0w / 2);
    for (int k = 0; k < FHW; ++k) {
      const int i = x0w + 2 * k, rx = region(i, d.nx);
      const bool ok = 2 * k < tb.tw + 2 * H;
      tb.col[k] = ok ? i : FUSED_NONE;
      tb.colrx[k] = rx;
      for (int ry = 0; ry < 3; ++ry)
        for (int p = 0; p < 2; ++p) {
          const int rb = R[ry][rx];
          if (!ok || rb < 0) continue;
          const BlockDev& B = lv.blk[rb];
          const int ii = local(i + p, rx, d.nx, B.nx);
          if (ii < 0 || ii >= B.nx) return fail(SNAC_ERR_INVALID_ARG, "fused window leaves its neighbour blocks");
          const Coef<double>& c = lv.cx[B.xo + ii];
          const PW<double>& w = lv.px[B.xo + ii];
          tb.xc[ry][p][k] = FP2<T>{(T)c.lo, (T)c.hi};
          tb.xd[ry][p][k] = (T)c.d;
          tb.px[ry][p][k] = FP2<T>{(T)w.self, (T)w.nbr};
        }
      if (2 * k >= H && 2 * k < H + tb.tw) {
        tb.rx[0][k] = (T)lv.rx[d.xo + i];
        tb.rx[1][k] = (T)lv.rx[d.xo + i + 1];
      }
    }
    for (int wj = 0; wj < FWN; ++wj) {
      const int j = y0w + wj, ry = region(j, d.ny);
      tb.rowry[wj] = ry;
      if (j >= 0 && j < d.ny) tb.ry[wj] = (T)lv.ry[d.yo + j];
      for (int rx = 0; rx < 3; ++rx) {
        const int rb = R[ry][rx];
        tb.rowoff[rx][wj] = FUSED_NONE;
        if (wj >= tb.th + 2 * H || rb < 0) continue;
        const BlockDev& B = lv.blk[rb];
        const int jj = local(j, ry, d.ny, B.ny);
        if (jj < 0 || jj >= B.ny) return fail(SNAC_ERR_INVALID_ARG, "fused window leaves its neighbour blocks");
        const Coef<double>& c = lv.cy[B.yo + jj];
        const PW<double>& w = lv.py[B.yo + jj];
        tb.yc[rx][wj] = FP2<T>{(T)c.lo, (T)c.hi};
        tb.yd[rx][wj] = (T)c.d;
        tb.py[rx][wj] = FP2<T>{(T)w.self, (T)w.nbr};
        const long long shift = rx == 0 ? B.nx : (rx == 2 ? -(long long)d.nx : 0);
        tb.rowoff[rx][wj] = (int)(B.off + (long long)jj * B.nx + shift);
      }
    }
    // coarse window: a column is kept where it lies inside every region block of its region column
    // (the columns the prolongation reads always do: they stay within 4 cells of the tile's block)
    const int cx0 = x0w / 2 - 1, cy0 = y0w / 2 - 1;
    for (int ci = 0; ci < FCW; ++ci) {
      const int I = cx0 + ci, rx = region(I, dc.nx);
      bool ok = true;
      for (int ry = 0; ry < 3; ++ry) {
        const int rb = R[ry][rx];
        if (rb < 0) continue;
        const int ii = local(I, rx, dc.nx, lc.blk[rb].nx);
        ok = ok && ii >= 0 && ii < lc.blk[rb].nx;
      }
      tb.ccol[ci] = ok ? I : FUSED_NONE;
      tb.ccolrx[ci] = rx;
    }
    for (int cj = 0; cj < FCW; ++cj) {
      const int J = cy0 + cj, ry = region(J, dc.ny);
      for (int rx = 0; rx < 3; ++rx) {
        const int rb = R[ry][rx];
        tb.crowoff[rx][cj] = FUSED_NONE;
        if (rb < 0) continue;
        const BlockDev& B = lc.blk[rb];
        const int jj = local(J, ry, dc.ny, B.ny);
        if (jj < 0 || jj >= B.ny) continue;
        const long long shift = rx == 0 ? B.nx : (rx == 2 ? -(long long)dc.nx : 0);
        tb.crowoff[rx][cj] = (int)(B.off + (long long)jj * B.nx + shift);
      }
    }
  }
  FusedTab<T>* d = nullptr;
  const int st = upload(P, &d, tabs);
  lv.d_ftab = d;
  return st;
}

// Caller axis of each internal axis: the two non-homogeneous axes in increasing order, then the
// homogeneous one (the plan works on internal (i, j) planes and transforms along internal k).
void axis_order(int homog, int (&perm)[3]) {
  int k = 0;
  for (int a = 0; a < 3; ++a)
    if (a != homog) perm[k++] = a;
  perm[2] = homog;
}

// The blocks with their axes in internal order (the cell-width arrays are shared, not copied).
std::vector<snac_block> internal_blocks(int nblocks, const snac_block* blocks, int homog) {
  int perm[3];
  axis_order(homog, perm);
  std::vector<snac_block> out(blocks, blocks + nblocks);
  for (int b = 0; b < nblocks; ++b)
    for (int a = 0; a < 3; ++a) {
      const int c = perm[a];
      out[b].lo[a] = blocks[b].lo[c];
      out[b].hi[a] = blocks[b].hi[c];
      out[b].h_dx[a] = blocks[b].h_dx[c];
      for (int sd = 0; sd < 2; ++sd) {
        out[b].bc[a][sd] = blocks[b].bc[c][sd];
        out[b].nbr[a][sd] = blocks[b].nbr[c][sd];
      }
    }
  return out;
}

int create(snac_plan** out, int32_t nblocks, const snac_block* blocks_in, int32_t homog_axis, const snac_options* opt) {
  if (!out || !blocks_in || nblocks < 1) return fail(SNAC_ERR_INVALID_ARG, "out/blocks NULL or nblocks < 1");
  *out = nullptr;
  if (homog_axis < 0 || homog_axis > 2) return fail(SNAC_ERR_INVALID_ARG, "homog_axis must be 0, 1 or 2");
  const std::vector<snac_block> iblocks = internal_blocks(nblocks, blocks_in, homog_axis);
  const snac_block* blocks = iblocks.data();
  std::vector<HBlock> hb;
  int st = validate(nblocks, blocks, hb);
  if (st) return st;
  snac_plan* P = new (std::nothrow) snac_plan();
  if (!P) return fail(SNAC_ERR_OOM, "host allocation");
  if (opt) {
    P->precision = opt->precision;
    P->nu1 = opt->nu1;
    P->nu2 = opt->nu2;
    P->max_outer = opt->max_outer;
    P->max_cycles = opt->max_cycles;
    P->max_coarse = opt->max_coarse;
    P->inner_reduction = opt->inner_reduction;
    P->fused = opt->fused;
    P->shift = opt->shift;
    P->onchip_opt = opt->onchip;
    if (opt->onchip != 0 && opt->onchip != -1) {
      delete P;
      return fail(SNAC_ERR_INVALID_ARG, "bad snac_options: onchip must be 0 or -1");
    }
    P->bottom_cells = opt->bottom_cells;
    if (opt->bottom_cells != 0 && opt->bottom_cells != -1 &&
        (opt->bottom_cells < 16 || opt->bottom_cells > BOTTOM_MAX_CELLS)) {
      delete P;
      return fail(SNAC_ERR_INVALID_ARG, "bad snac_options: bottom_cells must be 0, -1 or 16 .. 8192");
    }
    if (!(P->inner_reduction >= 0.0 && P->inner_reduction < 1.0) || !(P->shift <= 0.0) || !std::isfinite(P->shift) || (P->precision != SNAC_FP64 && P->precision != SNAC_MIXED) || P->nu1 < 0 || P->nu2 < 0 ||
        P->nu1 + P->nu2 < 1 || P->nu1 > 16 || P->nu2 > 16 || P->max_outer < 1 || P->max_cycles < 1 ||
        P->max_coarse < 1 || P->max_coarse > MAX_COARSE) {
      delete P;
      return fail(SNAC_ERR_INVALID_ARG, "bad snac_options");
    }
  }
  cudaGetDevice(&P->device);
  if (cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess || P->sms < 1) {
    cudaGetLastError();
    P->sms = 152;
  }
  P->nblk = nblocks;
  P->nzt = hb[0].n[2];
  P->nz = P->nzt;
  if (opt && (opt->mode_begin != 0 || opt->mode_end != 0)) {
    if (opt->mode_begin < 0 || opt->mode_end <= opt->mode_begin || opt->mode_end > P->nzt) {
      delete P;
      return fail(SNAC_ERR_INVALID_ARG, "mode_begin/mode_end must satisfy 0 <= mode_begin < mode_end <= n_z");
    }
    P->q0 = opt->mode_begin;
    P->nz = opt->mode_end - opt->mode_begin;
    P->ranged = true;
  }
  P->dz = hb[0].w[2][0];
  const int zl = hb[0].bc[2][0], zh = hb[0].bc[2][1];
  if (zl == SNAC_BC_PERIODIC) P->kind = KIND_PP;
  else if (zl == SNAC_BC_NEUMANN && zh == SNAC_BC_NEUMANN) P->kind = KIND_NN;
  else if (zl == SNAC_BC_DIRICHLET && zh == SNAC_BC_DIRICHLET) P->kind = KIND_DD;
  else if (zl == SNAC_BC_NEUMANN) P->kind = KIND_ND;
  else P->kind = KIND_DN;
  P->theta = P->kind == KIND_PP ? P->nzt : 2.0 * P->nzt;
  bool dirichlet_xy = false;
  for (const HBlock& h : hb)
    for (int a = 0; a < 2; ++a)
      for (int sd = 0; sd < 2; ++sd) dirichlet_xy |= h.bc[a][sd] == SNAC_BC_DIRICHLET;
  P->singular = (P->kind == KIND_PP || P->kind == KIND_NN) && !dirichlet_xy && P->shift == 0.0;
  const size_t inner = P->precision == SNAC_FP64 ? sizeof(double) : sizeof(float);
  long long off3 = 0;
  P->vol_total = 0.0;
  P->area_total = 0.0;
  for (const HBlock& h : hb) {
    P->blk_off3.push_back(off3);
    {
      // caller strides of the internal axes: the caller block is [z][y][x], x fastest
      int perm[3];
      axis_order(homog_axis, perm);
      long long n_caller[3], s_caller[3];
      for (int a = 0; a < 3; ++a) n_caller[perm[a]] = h.n[a];
      s_caller[0] = 1;
      s_caller[1] = n_caller[0];
      s_caller[2] = n_caller[0] * n_caller[1];
      P->cblk.push_back({off3, {s_caller[perm[0]], s_caller[perm[1]], s_caller[perm[2]]}});
    }
    off3 += (long long)h.n[0] * h.n[1] * h.n[2];
    double ax = 0, ay = 0;
    for (double w : h.w[0]) ax += w;
    for (double w : h.w[1]) ay += w;
    P->area_total += ax * ay;
  }
  P->n3 = off3;
  P->vol_total = P->area_total * P->dz * P->nzt;

  do {
    if ((st = build_levels(P, hb))) break;
    for (HostLevel& lv : P->lev)
      if ((st = upload_level(P, lv, inner))) break;
    if (st) break;
    // z operator pieces (uniform spacing). The ends are written as a mirrored ghost on the cell
    // itself: Neumann ghost = p_0 (coefficient +1/dz^2), Dirichlet ghost = -p_0 (-1/dz^2); the
    // diagonal is then -2/dz^2 on every plane, and carries the Helmholtz shift.
    const double iz2 = 1.0 / (P->dz * P->dz);
    for (int k = 0; k < P->nzt; ++k) {
      const bool per = P->kind == KIND_PP;
      Coef<double> c{iz2, iz2, -2.0 * iz2 + P->shift, P->dz};
      if (!per && k == 0) c.lo = zl == SNAC_BC_DIRICHLET ? -iz2 : iz2;
      if (!per && k == P->nzt - 1) c.hi = zh == SNAC_BC_DIRICHLET ? -iz2 : iz2;
      P->cz.push_back(c);
    }
    if ((st = upload(P, &P->d_cz, P->cz)) || (st = upload(P, &P->d_cblk, P->cblk))) break;
    {
      std::vector<float4> czff(P->nzt);
      for (int k = 0; k < P->nzt; ++k) {
        const float lh = (float)P->cz[k].lo, hh = (float)P->cz[k].hi;
        czff[k] = make_float4(lh, (float)(P->cz[k].lo - (double)lh), hh, (float)(P->cz[k].hi - (double)hh));
      }
      if ((st = upload(P, &P->d_czff, czff))) break;
      if (P->precision == SNAC_MIXED && !P->ranged) {
        auto pair = [](double v, float& h, float& l) {
          h = (float)v;
          l = (float)(v - (double)h);
        };
        const HostLevel& l0 = P->lev[0];
        std::vector<float4> cxf(l0.cx.size()), cyf(l0.cy.size());
        for (size_t i = 0; i < l0.cx.size(); ++i) {
          pair(l0.cx[i].lo, cxf[i].x, cxf[i].y);
          pair(l0.cx[i].hi, cxf[i].z, cxf[i].w);
        }
        for (size_t j = 0; j < l0.cy.size(); ++j) {
          pair(l0.cy[j].lo, cyf[j].x, cyf[j].y);
          pair(l0.cy[j].hi, cyf[j].z, cyf[j].w);
        }
        // the diagonal in the order the FP64 residual forms it: (cx.d + cy.d) + cz.d
        std::vector<float2> dgf(l0.ncell);
        for (const BlockDev& d : l0.blk)
          for (int j = 0; j < d.ny; ++j)
            for (int i = 0; i < d.nx; ++i) {
              const long long c = d.off + (long long)j * d.nx + i;
              pair(l0.cx[d.xo + i].d + l0.cy[d.yo + j].d + P->cz[0].d, dgf[c].x, dgf[c].y);
            }
        if ((st = upload(P, &P->d_cxff, cxf)) || (st = upload(P, &P->d_cyff, cyf)) || (st = upload(P, &P->d_dgff, dgf)))
          break;
      }
    }
    // the wavenumbers the plan holds: q0 .. q0 + nz - 1 of the n_z-point transform
    for (int l = 0; l < P->nz; ++l) {
      P->sigma.push_back(mode_lambda(P->kind, P->nzt, P->q0 + l) * iz2 + P->shift);
      P->pweight.push_back(parseval_weight(P->kind, P->nzt, P->q0 + l));
    }
    if ((st = upload(P, &P->d_sigma64, P->sigma)) || (st = upload(P, &P->d_sigma32, to32(P->sigma)))) break;
    if ((st = upload(P, &P->d_pweight, P->pweight))) break;
    std::vector<int> sm(P->nz, 0);
    for (int l = 0; l < P->nz; ++l) sm[l] = (P->singular && mode_lambda(P->kind, P->nzt, P->q0 + l) == 0.0) ? 1 : 0;
    if ((st = upload(P, &P->d_singular_mode, sm))) break;
    if ((st = build_coarse(P))) break;
    // the bottom of the cycle in one launch: from the first level below 0 whose planes, with all
    // coarser ones, fit in one CTA's shared memory (at least one smoothed level above the coarsest)
    // and whose plane has at most bottom_cells cells
    {
      const int L = (int)P->lev.size() - 1;
      const long long cap = P->bottom_cells > 0 ? P->bottom_cells : BOTTOM_MAX_CELLS;
      P->bottom = -1;
      if (P->nu1 >= 1 && P->nu2 >= 1 && P->bottom_cells != -1)
        for (int l = std::max(1, L - BOTTOM_MAX_LEVELS + 1); l < L; ++l)
          if (P->lev[l].ncell <= cap && L - l < BOTTOM_MAX_LEVELS &&
              bottom_layout(P, l, inner).bytes <= (size_t)BOTTOM_MAX_SMEM) {
            P->bottom = l;
            break;
          }
    }
    // the whole hierarchy on chip: every wavenumber's complete solve in one CTA (kern_bottom.cu)
    {
      const int L = (int)P->lev.size() - 1;
      P->onchip = P->onchip_opt == 0 && P->nu1 >= 1 && P->nu2 >= 1 && L >= 1 && L < BOTTOM_MAX_LEVELS &&
                  P->lev[0].ncell <= BOTTOM_MAX_CELLS && bottom_layout(P, 0, inner).bytes <= (size_t)BOTTOM_MAX_SMEM;
    }
    // the automatic inner reduction: an on-chip plan's V-cycles are cheap next to an outer step,
    // so it asks more of each step (measured on c64: 3 outer steps at 1e-4, 2 at 3e-5, 18 % faster)
    if (P->inner_reduction == 0.0) P->inner_reduction = P->onchip ? 3e-5 : 1e-4;
    // fused FP32 tile kernels on the levels whose blocks all keep the halo inside their neighbours
    // (above the bottom sub-cycle; not needed when the whole solve runs on chip)
    const bool want_fused = !P->onchip && (P->fused == 1 || (P->fused < 0 && P->precision == SNAC_MIXED));
    if (want_fused && P->nu1 >= 1 && P->nu2 >= 1 && P->nu1 <= 2 && P->nu2 <= 2) {
      for (size_t l = 0; l + 1 < P->lev.size(); ++l) {
        if (P->bottom >= 0 && (int)l >= P->bottom) break;
        HostLevel& lv = P->lev[l];
        bool ok = true;
        for (const BlockDev& d : lv.blk) ok = ok && d.nx >= FUSED_MIN_BLOCK && d.ny >= FUSED_MIN_BLOCK;
        if (!ok) continue;
        lv.fused = true;
        char* u2 = nullptr;
        if ((st = dmalloc(P, &u2, (size_t)P->nz * lv.ncell * inner))) break;
        lv.d_u2 = u2;
        for (int b = 0; b < lv.nblk; ++b)
          for (int y0 = 0; y0 < lv.blk[b].ny; y0 += FTILE_Y)
            for (int x0 = 0; x0 < lv.blk[b].nx; x0 += FTILE_X) lv.ftiles.push_back({b, x0, y0, 0});
        if (P->precision == SNAC_FP64) st = upload_fused_tabs<double>(P, lv, P->lev[l + 1]);
        else st = upload_fused_tabs<float>(P, lv, P->lev[l + 1]);
        if (st) break;
      }
      if (st) break;
    }
    if (P->precision == SNAC_FP64) {
      bool any_fused = false;
      for (const HostLevel& lv : P->lev) any_fused = any_fused || lv.fused;
      P->scaled_f = !any_fused && P->lev.size() > 1 && !P->onchip;
      for (size_t l = 0; l + 1 < P->lev.size(); ++l)
        if ((st = dmalloc(P, &P->lev[l].d_invd, (size_t)P->nz * P->lev[l].ncell))) break;
      if (st) break;
      // on a private non-blocking stream: plan creation does not wait for other streams' work
      cudaStream_t cs = nullptr;
      bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
      ok = ok && launch_inverse_diagonals(P, cs) == cudaSuccess && cudaStreamSynchronize(cs) == cudaSuccess;
      if (cs) cudaStreamDestroy(cs);
      if (!ok) {
        st = fail(SNAC_ERR_CUDA, "computing the inverse diagonals failed");
        break;
      }
    }
    if (P->bottom > 0) {  // the bottom sub-cycle's level table (after the inverse diagonals exist)
      const int L = (int)P->lev.size() - 1;
      auto build_bottom = [&](auto tag) -> int {
        using T = decltype(tag);
        const BottomLayout lay = bottom_layout(P, P->bottom, sizeof(T));
        std::vector<BottomLevel<T>> tab;
        for (int l = P->bottom; l <= L; ++l) {
          const int k = l - P->bottom;
          BottomLevel<T> b{};
          b.L = level_view<T>(P->lev[l]);
          b.invd = (sizeof(T) == 8 && l < L) ? P->lev[l].d_invd : nullptr;
          b.su = lay.su[k];
          b.sf = lay.sf[k];
          b.sinv = lay.sinv[k];
          b.sblk = lay.sblk[k];
          tab.push_back(b);
        }
        BottomLevel<T>* d = nullptr;
        const int s2 = upload(P, &d, tab);
        P->d_bottom = d;
        return s2;
      };
      if ((st = P->precision == SNAC_FP64 ? build_bottom(double{}) : build_bottom(float{}))) break;
    }
    if (P->onchip) {  // the same kind of table for the whole hierarchy, from level 0
      const int L = (int)P->lev.size() - 1;
      auto build_onchip = [&](auto tag) -> int {
        using T = decltype(tag);
        const BottomLayout lay = bottom_layout(P, 0, sizeof(T));
        std::vector<BottomLevel<T>> tab;
        for (int l = 0; l <= L; ++l) {
          BottomLevel<T> b{};
          b.L = level_view<T>(P->lev[l]);
          b.invd = (sizeof(T) == 8 && l < L) ? P->lev[l].d_invd : nullptr;
          b.su = lay.su[l];
          b.sf = lay.sf[l];
          b.sinv = lay.sinv[l];
          b.sblk = lay.sblk[l];
          tab.push_back(b);
        }
        BottomLevel<T>* d = nullptr;
        const int s2 = upload(P, &d, tab);
        P->d_onchip = d;
        return s2;
      };
      if ((st = P->precision == SNAC_FP64 ? build_onchip(double{}) : build_onchip(float{}))) break;
    }
    if ((st = build_twiddles(P))) break;
    P->tc64 = transform_columns(P->nzt, true);
    P->tc32 = transform_columns(P->nzt, false);
    if ((st = build_chunks(P, P->tc64, P->chunks64, &P->d_chunks64))) break;
    if ((st = build_chunks(P, P->tc32, P->chunks32, &P->d_chunks32))) break;
    {
      const HostLevel& l0 = P->lev[0];
      std::vector<double> area(l0.ncell);
      for (const BlockDev& d : l0.blk)
        for (int j = 0; j < d.ny; ++j)
          for (int i = 0; i < d.nx; ++i) area[d.off + (long long)j * d.nx + i] = l0.cx[d.xo + i].w * l0.cy[d.yo + j].w;
      if ((st = upload(P, &P->d_area0, area))) break;
    }
    if (!P->ranged && (st = dmalloc(P, &P->d_r3, (size_t)P->n3))) break;
    const int zsplit = std::min(P->nzt, 16);
    // per-CTA partial sums: the 3-D residual grid (tiles x z split) or a plane reduction (MEAN_CTAS)
    P->npartial = std::max((int)P->lev[0].tiles.size() * zsplit, MEAN_CTAS);
    if ((st = dmalloc(P, &P->d_partial, (size_t)P->npartial * 4))) break;
    if ((st = dmalloc(P, &P->d_sums, SUM_SLOTS)) || (st = dmalloc(P, &P->d_flag, 1))) break;
    // per-mode, per-tile partial sums (basic tiles; the fused tiles are fewer)
    if ((st = dmalloc(P, &P->d_mode_part, (size_t)P->nz * std::max<size_t>(P->lev[0].tiles.size(), 64)))) break;
    if ((st = dmalloc(P, &P->d_mode_norm2, (size_t)P->nz))) break;
    if (P->onchip && (st = dmalloc(P, &P->d_fused, 2))) break;
    if ((st = dmalloc(P, &P->d_active, (size_t)P->nz)) || (st = dmalloc(P, &P->d_check, (size_t)P->nz))) break;
    auto mapped = [](auto** h, auto** dh, size_t n) {
      return cudaHostAlloc((void**)h, n * sizeof(**h), cudaHostAllocMapped) == cudaSuccess &&
             cudaHostGetDevicePointer((void**)dh, (void*)*h, 0) == cudaSuccess;
    };
    if (!mapped(&P->h_sums, &P->dh_sums, SUM_SLOTS) || !mapped(&P->h_mode_norm2, &P->dh_mode_norm2, P->nz) ||
        !mapped(&P->h_active, &P->dh_active, P->nz) || !mapped(&P->h_check, &P->dh_check, P->nz) ||
        !mapped(&P->h_cycles, &P->dh_cycles, P->nz) || !mapped(&P->h_wait, &P->dh_wait, 1)) {
      st = fail(SNAC_ERR_OOM, "pinned host allocation");
      break;
    }
    {
      // the pre-pass flag starts at zero (its reduction resets it after each use); on a private
      // non-blocking stream, like every other device write of plan creation
      cudaStream_t cs = nullptr;
      bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
                cudaMemsetAsync(P->d_flag, 0, sizeof(int), cs) == cudaSuccess && cudaStreamSynchronize(cs) == cudaSuccess;
      if (cs) cudaStreamDestroy(cs);
      if (!ok) {
        st = fail(SNAC_ERR_CUDA, "initialising the pre-pass flag failed");
        break;
      }
    }
  } while (0);
  if (st) {
    free_plan(P);
    return st;
  }
  P->mode_cycles.assign(P->nz, 0);
  P->info.levels = (int)P->lev.size();
  P->info.n_modes = P->nz;
  *out = P;
  return SNAC_OK;
}

}  // namespace

namespace snac {
int plan_inner_size(const snac_plan* P) { return P->precision == SNAC_FP64 ? 8 : 4; }

int check_layout(int nblocks, const snac_block* blocks, int homog_axis) {
  if (!blocks || nblocks < 1) return fail(SNAC_ERR_INVALID_ARG, "blocks NULL or nblocks < 1");
  if (homog_axis < 0 || homog_axis > 2) return fail(SNAC_ERR_INVALID_ARG, "homog_axis must be 0, 1 or 2");
  const std::vector<snac_block> ib = internal_blocks(nblocks, blocks, homog_axis);
  std::vector<HBlock> hb;
  return validate(nblocks, ib.data(), hb);
}
}  // namespace snac

extern "C" {

int snac_plan_create(snac_plan** out, int32_t nblocks, const snac_block* blocks, int32_t homog_axis,
                     const snac_options* opt) {
  try {
    return create(out, nblocks, blocks, homog_axis, opt);
  } catch (...) {
    return fail(SNAC_ERR_OOM, "exception during plan creation");
  }
}

int snac_plan_workspace_bytes(const snac_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return SNAC_ERR_INVALID_ARG;
  *bytes = plan->bytes;
  return SNAC_OK;
}

int snac_plan_info(const snac_plan* plan, snac_solve_info* info) {
  if (!plan || !info) return SNAC_ERR_INVALID_ARG;
  *info = plan->info;
  return SNAC_OK;
}

int snac_plan_mode_cycles(const snac_plan* plan, int32_t* h_cycles, int32_t n) {
  if (!plan || !h_cycles || n < plan->nz) return SNAC_ERR_INVALID_ARG;
  std::copy(plan->mode_cycles.begin(), plan->mode_cycles.end(), h_cycles);
  return SNAC_OK;
}

int snac_plan_destroy(snac_plan* plan) {
  free_plan(plan);
  return SNAC_OK;
}

const char* snac_status_string(int status) {
  switch (status) {
    case SNAC_OK: return "ok";
    case SNAC_ERR_INVALID_ARG: return "invalid argument";
    case SNAC_ERR_LAYOUT: return "invalid block layout";
    case SNAC_ERR_OOM: return "out of memory";
    case SNAC_ERR_CUDA: return "CUDA error";
    case SNAC_ERR_NOT_CONVERGED: return "not converged";
    case SNAC_ERR_NONFINITE: return "non-finite residual";
    case SNAC_ERR_INCOMPATIBLE_RHS: return "incompatible right-hand side";
    case SNAC_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* snac_last_error_message(void) { return snac::g_last_error.c_str(); }

}  // extern "C"
