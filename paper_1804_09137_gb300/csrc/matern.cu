// Matérn covariance generation (Sec. IV, eq. 5) on the device.
//
// K_nu, K_(nu-1) and dK_nu/dnu come from the integral representation
//   K_mu(x) = int_0^inf exp(-x cosh t) cosh(mu t) dt          (DLMF 10.32.9)
//   dK_nu/dnu(x) = int_0^inf t sinh(nu t) exp(-x cosh t) dt
// evaluated by the trapezoidal rule, which converges geometrically for this
// analytic, doubly exponentially decaying integrand (step h = min(0.1, 0.5/sqrt x),
// cut where x cosh t > 750).  With them, for x = r / beta and c_nu = 1/(2^(nu-1) Gamma(nu)):
//   C        = sigma2 c_nu x^nu K_nu(x)
//   dC/dbeta = sigma2 c_nu x^(nu+1) K_(nu-1)(x) / beta
//   dC/dnu   = C (ln x - ln 2 - psi(nu)) + sigma2 c_nu x^nu dK_nu/dnu(x).
// These exact values are taken at the Chebyshev nodes of 176 geometric
// intervals covering [2^-44 r_max, r_max] (four per octave) and turned into
// degree-12 polynomials, so that generating an entry costs one table lookup
// and 12 FMAs instead of a Bessel evaluation (float64 is the scarce pipe on
// this GPU).  Interpolation error is below 1e-14 of sigma2 (tested against the
// scipy-based oracle).
#include <math.h>

#include "common.cuh"
#include "df.cuh"

namespace {

__device__ void matern_direct_warp(double r, const MaternParams mp, double* f0, double* f1, double* f2) {
  const int lane = threadIdx.x & 31;
  const double x = r / mp.beta;
  const double h = fmin(0.1, 0.5 / sqrt(x));
  const double tmax = acosh(fmax(750.0 / x, 1.0)) + 2.0;
  const int N = (int)ceil(tmax / h);
  const double nu = mp.nu;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int m = lane; m <= N; m += 32) {
    const double t = m * h;
    const double w = (m == 0) ? 0.5 * h : h;
    const double e = w * exp(-x * cosh(t));
    s0 += e * cosh(nu * t);
    s1 += e * cosh((nu - 1.0) * t);
    s2 += e * t * sinh(nu * t);
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  const double xnu = pow(x, nu);
  const double base = mp.sigma2 * mp.cnu * xnu;
  const double C = base * s0;
  *f0 = C;
  *f1 = base * x * s1 / mp.beta;
  *f2 = C * (log(x) - 0.69314718055994530942 - mp.psi) + base * s2;
}

// one warp per (interval, node): exact values at the Chebyshev nodes
__global__ void k_tab_nodes(const MaternParams mp, double* __restrict__ vals) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= TAB_NINT * TAB_NC) return;
  const int j = gw / TAB_NC, m = gw % TAB_NC;
  const int oct = j / TAB_SUB, q = j % TAB_SUB;
  const double edges[5] = {1.0, 1.18920711500272106672, 1.41421356237309504880, 1.68179283050742908606, 2.0};
  const double a = edges[q], b = edges[q + 1];
  const double tn = cos(3.14159265358979323846 * (m + 0.5) / TAB_NC);
  const double r = ldexp(0.5 * (a + b) + 0.5 * (b - a) * tn, mp.e_lo + oct);
  double f0, f1, f2;
  matern_direct_warp(r, mp, &f0, &f1, &f2);
  if ((threadIdx.x & 31) == 0) {
    vals[(0 * TAB_NINT + j) * TAB_NC + m] = f0;
    vals[(1 * TAB_NINT + j) * TAB_NC + m] = f1;
    vals[(2 * TAB_NINT + j) * TAB_NC + m] = f2;
  }
}

// one thread per (function, interval): Chebyshev coefficients -> monomial in t
__global__ void k_tab_coefs(const double* __restrict__ vals, double* __restrict__ tab) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= TAB_NFUN * TAB_NINT) return;
  const double* v = vals + (size_t)id * TAB_NC;
  double c[TAB_NC];
  for (int l = 0; l < TAB_NC; ++l) {
    double s = 0.0;
    for (int m = 0; m < TAB_NC; ++m) s += v[m] * cos(3.14159265358979323846 * l * (m + 0.5) / TAB_NC);
    c[l] = (l == 0 ? 1.0 : 2.0) * s / TAB_NC;
  }
  double a[TAB_NC], Tm[TAB_NC], T0[TAB_NC], T1[TAB_NC];
  for (int d = 0; d < TAB_NC; ++d) { a[d] = 0.0; T0[d] = 0.0; T1[d] = 0.0; }
  T0[0] = 1.0;
  T1[1] = 1.0;
  a[0] += c[0];
  for (int d = 0; d < TAB_NC; ++d) a[d] += c[1] * T1[d];
  for (int l = 2; l < TAB_NC; ++l) {
    for (int d = 0; d < TAB_NC; ++d) Tm[d] = (d > 0 ? 2.0 * T1[d - 1] : 0.0) - T0[d];
    for (int d = 0; d < TAB_NC; ++d) { a[d] += c[l] * Tm[d]; T0[d] = T1[d]; T1[d] = Tm[d]; }
  }
  double* out = tab + (size_t)id * TAB_NC;
  for (int d = 0; d < TAB_NC; ++d) out[d] = a[d];
}

__global__ void k_gen_diag(const double* __restrict__ tab, const MaternParams mp, const double* __restrict__ x,
                           const double* __restrict__ y, int64_t n, int nb, double* __restrict__ D) {
  const int k = blockIdx.y;
  const int64_t nn = (int64_t)nb * nb;
  double* Dk = D + (size_t)k * nn;
  const int64_t base = (int64_t)k * nb;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < nn; id += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(id % nb), b = (int)(id / nb);
    Dk[id] = cov_pts(tab, mp, x, y, n, base + a, base + b);
  }
}

// the coefficients as double-float pairs (bit conversion; magnitudes below 2^-126 become zero)
__global__ void k_tab_df(const double* __restrict__ tab, float2* __restrict__ tabf) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id < TAB_ELEMS) tabf[id] = df_from_scaled(tab[id], 0);
}

}  // namespace

int tlr_build_table(tlr_ctx* h, cudaStream_t s) {
  double* vals = h->scratch;  // TAB_ELEMS doubles of workspace
  const int warps = TAB_NINT * TAB_NC;
  k_tab_nodes<<<(warps * 32 + 255) / 256, 256, 0, s>>>(h->mp, vals);
  TLR_LAUNCH_CHECK();
  k_tab_coefs<<<(TAB_NFUN * TAB_NINT + 127) / 128, 128, 0, s>>>(vals, h->tab);
  TLR_LAUNCH_CHECK();
  if (h->tabf) {
    k_tab_df<<<(TAB_ELEMS + 255) / 256, 256, 0, s>>>(h->tab, h->tabf);
    TLR_LAUNCH_CHECK();
  }
  h->tab_valid = 1;
  return TLR_OK;
}

int tlr_gen_diag(tlr_ctx* h, cudaStream_t s) {
  dim3 grid(64, h->nt);
  k_gen_diag<<<grid, 256, 0, s>>>(h->tab, h->mp, h->x, h->y, h->n, h->nb, h->D);
  TLR_LAUNCH_CHECK();
  return TLR_OK;
}

