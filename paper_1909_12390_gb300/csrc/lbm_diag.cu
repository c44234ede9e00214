// Device-side diagnostics of a two-phase state (Section 4.2 and Section 4.3 checks): the
// rho = (rho_max + rho_min) / 2 contour of the total density, the bulk phases (cells farther
// than a given distance from the contour), their mean component densities, pressures and
// molar compositions, the iso-fugacity residual of Eq. error evaluated from the bulk states
// (Z = p / (n R T), no cubic solve), the liquid volume, the equivalent radius and the
// pressure jump of Laplace's law.
//
// Distance to the contour is measured in the L-infinity norm: a cell is bulk liquid when every
// cell of the (2e + 1)^D box around it (periodic) lies above the contour level, bulk vapour
// when every one lies below. The box contains the Euclidean ball of radius e, so these cells
// are at least e away from the contour in the Euclidean sense too.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "lbm.h"
#include "lbm_host.h"

namespace {

constexpr double kSqrt2 = 1.4142135623730950488;

// total density per site and its extreme values (bit patterns of positive doubles order like
// the values); mx/mn start at 0 / all ones
__global__ void k_total(const double* __restrict__ rho, long long N, int nc, double* __restrict__ tot,
                        unsigned long long* mx, unsigned long long* mn) {
  unsigned long long lmx = 0, lmn = ~0ull;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < nc; ++c) t += rho[c * N + i];
    tot[i] = t;
    const unsigned long long b = (unsigned long long)__double_as_longlong(t);
    lmx = max(lmx, b);
    lmn = min(lmn, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lmx = max(lmx, __shfl_xor_sync(0xffffffffu, lmx, o));
    lmn = min(lmn, __shfl_xor_sync(0xffffffffu, lmn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(mx, lmx);
    atomicMin(mn, lmn);
  }
}

__global__ void k_mask(const double* __restrict__ tot, long long N, double thr, unsigned char* all,
                       unsigned char* any) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const unsigned char v = tot[i] > thr ? 1 : 0;
    all[i] = v;
    any[i] = v;
  }
}

// One axis of the box erosion: out_all = min, out_any = max over |d| <= e along axis (periodic).
__global__ void k_erode_axis(const unsigned char* __restrict__ all, const unsigned char* __restrict__ any,
                             unsigned char* __restrict__ oall, unsigned char* __restrict__ oany, int nx, int ny,
                             int nz, int axis, int e) {
  const long long N = (long long)nx * ny * nz;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
    const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const int p = axis == 0 ? x : (axis == 1 ? y : z);
    const long long stride = axis == 0 ? 1 : (axis == 1 ? nx : (long long)nx * ny);
    const long long base = i - (long long)p * stride;
    unsigned char a = 1, b = 0;
    const int w = e < n ? e : n;  // a window longer than the axis covers it once
    for (int d = -w; d <= w; ++d) {
      int q = (p + d) % n;
      if (q < 0) q += n;
      a &= all[base + q * stride];
      b |= any[base + q * stride];
    }
    oall[i] = a;
    oany[i] = b;
  }
}

// sums[0..nc) liquid bulk rho_c, [nc] liquid bulk p, [nc+1] liquid bulk cells, then the same
// for the vapour bulk, then [2(nc+2)] cells above the contour
__global__ void k_bulk_sums(const double* __restrict__ rho, const double* __restrict__ p, long long N, int nc,
                            const unsigned char* __restrict__ all, const unsigned char* __restrict__ any,
                            const double* __restrict__ tot, double thr, double* sums) {
  double s[2 * (4 + 2) + 1];
  for (int k = 0; k < 2 * (nc + 2) + 1; ++k) s[k] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int ph = all[i] ? 0 : (any[i] ? -1 : 1);
    if (ph >= 0) {
      const int o = ph * (nc + 2);
      for (int c = 0; c < nc; ++c) s[o + c] += rho[c * N + i];
      s[o + nc] += p[i];
      s[o + nc + 1] += 1.0;
    }
    if (tot[i] > thr) s[2 * (nc + 2)] += 1.0;
  }
  for (int k = 0; k < 2 * (nc + 2) + 1; ++k) {
    double v = s[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&sums[k], v);
  }
}

// ln phi_i of Eq. fugacitycoeff2 at molar densities n_i and pressure p, with Z = p / (n R T)
void ln_phi_of_state(const lbm::Params& P, int nc, const double* n, double p, double* out) {
  double nt = 0.0;
  for (int i = 0; i < nc; ++i) nt += n[i];
  const double pr = p / P.RT, pr2 = pr / P.RT;  // p / RT and p / (RT)^2
  const double Z = p / (nt * P.RT);
  double c[4], s[4], A = 0.0, B = 0.0;
  for (int i = 0; i < nc; ++i) c[i] = n[i] / nt;
  for (int i = 0; i < nc; ++i) {
    s[i] = 0.0;
    for (int j = 0; j < nc; ++j) s[i] += P.Qa[i * 4 + j] * pr2 * c[j];
    A += c[i] * s[i];
    B += c[i] * P.b[i] * pr;
  }
  const double lg = std::log((Z + (1.0 - kSqrt2) * B) / (Z + (1.0 + kSqrt2) * B));
  for (int i = 0; i < nc; ++i) {
    const double Bi = P.b[i] * pr;
    out[i] = -std::log(Z - B) + Bi / B * (Z - 1.0) + A / (2.0 * kSqrt2 * B) * (2.0 * s[i] / A - Bi / B) * lg;
  }
}

}  // namespace

namespace lbm {

// The diagnostics on the state in rho (nc * N component densities) and p (N EOS pressures),
// device arrays; work is a device buffer of at least N doubles + 4 N bytes + 64 doubles.
lbm_status diagnostics(const Params& P, int nc, int D, const lbm_diag_params* dp, const double* rho,
                       const double* p, void* work, cudaStream_t s, lbm_diag_result* out, std::string* why) {
  const long long N = (long long)P.N;
  double* tot = (double*)work;
  unsigned char* m = (unsigned char*)(tot + N);  // 4 masks of N bytes
  double* small = (double*)(m + 4 * N + ((8 - (4 * N) % 8) % 8));
  unsigned long long* ext = (unsigned long long*)small;  // [0] max, [1] min
  double* sums = small + 2;
  const unsigned nb = (unsigned)std::min<long long>((N + 255) / 256, 2048);
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && why) *why = cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  if (!ck(cudaMemsetAsync(ext, 0, sizeof(unsigned long long), s)) ||
      !ck(cudaMemsetAsync(ext + 1, 0xff, sizeof(unsigned long long), s)) ||
      !ck(cudaMemsetAsync(sums, 0, 16 * sizeof(double), s)))
    return LBM_ERR_CUDA;
  k_total<<<nb, 256, 0, s>>>(rho, N, nc, tot, ext, ext + 1);
  unsigned long long hext[2];
  if (!ck(cudaGetLastError()) || !ck(cudaMemcpyAsync(hext, ext, sizeof hext, cudaMemcpyDeviceToHost, s)) ||
      !ck(cudaStreamSynchronize(s)))
    return LBM_ERR_CUDA;
  double mx, mn;
  std::memcpy(&mx, &hext[0], sizeof mx);
  std::memcpy(&mn, &hext[1], sizeof mn);
  const double thr = dp->threshold > 0 ? dp->threshold : 0.5 * (mx + mn);
  unsigned char *a0 = m, *b0 = m + N, *a1 = m + 2 * N, *b1 = m + 3 * N;
  k_mask<<<nb, 256, 0, s>>>(tot, N, thr, a0, b0);
  for (int ax = 0; ax < D; ++ax) {
    k_erode_axis<<<nb, 256, 0, s>>>(a0, b0, a1, b1, P.nx, P.ny, P.nz, ax, dp->erode);
    std::swap(a0, a1);
    std::swap(b0, b1);
  }
  k_bulk_sums<<<nb, 256, 0, s>>>(rho, p, N, nc, a0, b0, tot, thr, sums);
  double hs[2 * (4 + 2) + 1];
  if (!ck(cudaGetLastError()) ||
      !ck(cudaMemcpyAsync(hs, sums, (2 * (nc + 2) + 1) * sizeof(double), cudaMemcpyDeviceToHost, s)) ||
      !ck(cudaStreamSynchronize(s)))
    return LBM_ERR_CUDA;
  lbm_diag_result r{};
  r.threshold = thr;
  r.rho_max = mx;
  r.rho_min = mn;
  r.n_l = (int64_t)hs[nc + 1];
  r.n_v = (int64_t)hs[2 * nc + 3];
  const double nl = hs[nc + 1], nv = hs[2 * nc + 3];
  double ml[4] = {0, 0, 0, 0}, mv[4] = {0, 0, 0, 0};
  for (int c = 0; c < nc; ++c) {
    r.rho_l[c] = nl > 0 ? hs[c] / nl : NAN;
    r.rho_v[c] = nv > 0 ? hs[nc + 2 + c] / nv : NAN;
    ml[c] = r.rho_l[c] * P.invM[c];
    mv[c] = r.rho_v[c] * P.invM[c];
  }
  r.p_l = nl > 0 ? hs[nc] / nl : NAN;
  r.p_v = nv > 0 ? hs[2 * nc + 2] / nv : NAN;
  double sl = 0, sv = 0;
  for (int c = 0; c < nc; ++c) {
    sl += ml[c];
    sv += mv[c];
  }
  for (int c = 0; c < nc; ++c) {
    r.x[c] = ml[c] / sl;
    r.y[c] = mv[c] / sv;
  }
  r.residual = NAN;
  if (nl > 0 && nv > 0) {
    double lpl[4], lpv[4];
    ln_phi_of_state(P, nc, ml, r.p_l, lpl);
    ln_phi_of_state(P, nc, mv, r.p_v, lpv);
    double res = 0.0;
    for (int c = 0; c < nc; ++c) {
      const double q = std::exp(lpl[c] - lpv[c]) * r.x[c] * r.p_l / (r.y[c] * r.p_v) - 1.0;
      res += q * q;
    }
    r.residual = res;
  }
  r.liquid_cells = (int64_t)hs[2 * (nc + 2)];
  const double V = hs[2 * (nc + 2)];
  r.radius = D == 2 ? std::sqrt(V / (M_PI * P.nz)) : std::cbrt(3.0 * V / (4.0 * M_PI));
  r.dp = r.p_l - r.p_v;
  *out = r;
  return LBM_OK;
}

}  // namespace lbm
