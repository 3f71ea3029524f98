// Search parameters (Sec. 2.2): the velocity-set size, the number of
// independent stacks, the noise-peak statistics of a PSF-detected catalog and
// the threshold N_min that a false-positive budget requires, the per-epoch
// probability that a real source lands in its bin.  Host code only.
//
// Noise peaks: white sky noise under a Gaussian window of width a is a 2-D
// Gaussian field with gamma = 1/sqrt(2) and sigma2^2 / sigma1^2 = 2 / a^2.  By
// the Kac-Rice formula its maxima at height z have surface density
//   n(z) = phi(z) * (2 / (pi a^2)) * E[(T^2 - D^2)/4 ; T > D | z]
// (in units of sigma2: Hessian trace T ~ N(gamma z, 1 - gamma^2), anisotropy D
// Rayleigh with density 2 d exp(-d^2)).  The expectation over T has the closed
// form used below; the one over D and the integral over z are composite
// Gauss-Legendre sums.
#include <cmath>
#include <vector>

#include "sas_internal.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;
const double kGamma = 1.0 / std::sqrt(2.0);

double normal_pdf(double x) { return std::exp(-0.5 * x * x) / std::sqrt(2.0 * kPi); }
double normal_sf(double x) { return 0.5 * std::erfc(x / std::sqrt(2.0)); }

// E[(T^2 - D^2) 1{T > d}] for T ~ N(mu, s^2) at D = d:
// (mu^2 + s^2 - d^2) Q(c) + s (mu + d) phi(c), c = (d - mu) / s.
double trace_moment(double mu, double s, double d) {
  const double c = (d - mu) / s;
  return (mu * mu + s * s - d * d) * normal_sf(c) + s * (mu + d) * normal_pdf(c);
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton's method on P_n from its
// three-term recurrence).
struct GaussLegendre {
  static constexpr int n = 8;
  double x[n], w[n];
  GaussLegendre() {
    for (int i = 0; i < n; ++i) {
      double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

// Composite Gauss-Legendre over `panels` equal panels.
template <typename F>
double integrate(F f, double lo, double hi, int panels) {
  static const GaussLegendre gl;
  const double h = (hi - lo) / panels;
  double acc = 0.0;
  for (int p = 0; p < panels; ++p) {
    const double c = lo + (p + 0.5) * h;
    for (int i = 0; i < GaussLegendre::n; ++i) acc += gl.w[i] * f(c + 0.5 * h * gl.x[i]);
  }
  return acc * 0.5 * h;
}

double peak_density(double z, double a) {
  const double mu = kGamma * z, s = std::sqrt(1.0 - kGamma * kGamma);
  const double e = integrate([&](double d) { return 2.0 * d * std::exp(-d * d) * 0.25 * trace_moment(mu, s, d); },
                             0.0, 9.0, 48);
  return normal_pdf(z) * (2.0 / (kPi * a * a)) * e;
}

double peaks_above(double nu_th, double a) {
  const double hi = std::fmax(nu_th, 0.0) + 14.0;
  return integrate([&](double z) { return peak_density(z, a); }, nu_th, hi, 96);
}

double poisson_sf(uint32_t k, double lam) {
  if (k == 0) return 1.0;
  if (lam == 0.0) return 0.0;
  auto pmf = [&](double j) { return std::exp(-lam + j * std::log(lam) - std::lgamma(j + 1.0)); };
  if ((double)k > lam) {
    double total = 0.0;
    for (double j = k;; j += 1.0) {
      const double t = pmf(j);
      total += t;
      if (t == 0.0 || (t < total * 1e-17 && j > lam)) break;  // terms only shrink past lam
    }
    return total;
  }
  double below = 0.0;
  for (uint32_t j = 0; j < k; ++j) below += pmf((double)j);
  return 1.0 - below;
}

// Smallest k with P(N >= k) <= eps: P(N >= k) falls with k, so a binary search
// over [0, hi], hi far enough into the tail that it holds there.
uint32_t choose_n_min(double lam, double eps) {
  if (poisson_sf(0, lam) <= eps) return 0;
  uint32_t lo = 0, hi = (uint32_t)(lam + 60.0 * std::sqrt(lam) + 1000.0);  // sf(hi) < 1e-300
  while (hi - lo > 1) {  // sf(lo) > eps >= sf(hi)
    const uint32_t mid = lo + (hi - lo) / 2;
    if (poisson_sf(mid, lam) > eps) lo = mid; else hi = mid;
  }
  return hi;
}

double p_signal(double nu, double nu_th, double a, double dx) {
  const double in = std::erf(dx * nu / (4.0 * a));
  return 0.5 * std::erfc((nu_th - nu) / std::sqrt(2.0)) * in * in;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

using sas::set_error;

extern "C" {

int sas_param_velocity_count(double vmin_x, double vmax_x, double vmin_y, double vmax_y, double dx, double dt,
                             double* out) {
  if (!out) return set_error(SAS_ERR_ARG, "null output");
  if (!finite_pos(dx) || !finite_pos(dt) || !(vmax_x >= vmin_x) || !(vmax_y >= vmin_y))
    return set_error(SAS_ERR_ARG, "need dx > 0, dt > 0 and ordered velocity ranges");
  const double dv = dx / dt;
  *out = ((vmax_x - vmin_x) / dv) * ((vmax_y - vmin_y) / dv);
  return SAS_OK;
}

int sas_param_n_stacks(double n_velocities, double omega, double dx, double* out) {
  if (!out) return set_error(SAS_ERR_ARG, "null output");
  if (!(n_velocities >= 0) || !(omega >= 0) || !finite_pos(dx)) return set_error(SAS_ERR_ARG, "bad argument");
  *out = n_velocities * omega / (dx * dx);
  return SAS_OK;
}

int sas_param_peak_density(double z, double a, double* out) {
  if (!out) return set_error(SAS_ERR_ARG, "null output");
  if (!std::isfinite(z) || !finite_pos(a)) return set_error(SAS_ERR_ARG, "need finite z and a > 0");
  *out = peak_density(z, a);
  return SAS_OK;
}

int sas_param_peaks_above(double nu_th, double a, double* out) {
  if (!out) return set_error(SAS_ERR_ARG, "null output");
  if (!std::isfinite(nu_th) || !finite_pos(a)) return set_error(SAS_ERR_ARG, "need finite nu_th and a > 0");
  *out = peaks_above(nu_th, a);
  return SAS_OK;
}

int sas_param_noise_rate(double nu_th, const double* a, uint32_t n_epochs, double dx, double* out) {
  if (!out || (n_epochs && !a)) return set_error(SAS_ERR_ARG, "null argument");
  if (!std::isfinite(nu_th) || !finite_pos(dx)) return set_error(SAS_ERR_ARG, "need finite nu_th and dx > 0");
  for (uint32_t i = 0; i < n_epochs; ++i)
    if (!finite_pos(a[i])) return set_error(SAS_ERR_ARG, "PSF widths must be > 0");
  const double lam1 = peaks_above(nu_th, 1.0);
  double r = 0.0;
  for (uint32_t i = 0; i < n_epochs; ++i) r += lam1 * (dx / a[i]) * (dx / a[i]);
  *out = r;
  return SAS_OK;
}

int sas_param_poisson_sf(uint32_t k, double lambda, double* out) {
  if (!out) return set_error(SAS_ERR_ARG, "null output");
  if (!std::isfinite(lambda) || lambda < 0) return set_error(SAS_ERR_ARG, "need lambda >= 0");
  *out = poisson_sf(k, lambda);
  return SAS_OK;
}

int sas_param_choose_n_min(double lambda, double eps, uint32_t* out) {
  if (!out) return set_error(SAS_ERR_ARG, "null output");
  if (!std::isfinite(lambda) || lambda < 0 || !(eps > 0)) return set_error(SAS_ERR_ARG, "need lambda >= 0, eps > 0");
  if (lambda > 1e7) return set_error(SAS_ERR_RANGE, "lambda above 1e7");
  *out = choose_n_min(lambda, eps);
  return SAS_OK;
}

int sas_param_p_signal(double nu, double nu_th, double a, double dx, double* out) {
  if (!out) return set_error(SAS_ERR_ARG, "null output");
  if (!std::isfinite(nu) || !std::isfinite(nu_th) || !finite_pos(a) || !(dx >= 0))
    return set_error(SAS_ERR_ARG, "bad argument");
  *out = p_signal(nu, nu_th, a, dx);
  return SAS_OK;
}

int sas_param_signal_tail(const double* p, uint32_t n, uint32_t k, double* out) {
  if (!out || (n && !p)) return set_error(SAS_ERR_ARG, "null argument");
  if (n > 65536) return set_error(SAS_ERR_RANGE, "more than 65536 epochs");
  std::vector<double> dist(1, 1.0);
  for (uint32_t i = 0; i < n; ++i) {
    if (!(p[i] >= 0.0 && p[i] <= 1.0)) return set_error(SAS_ERR_ARG, "probabilities must lie in [0, 1]");
    std::vector<double> nxt(dist.size() + 1, 0.0);
    for (size_t j = 0; j < dist.size(); ++j) {
      nxt[j] += dist[j] * (1.0 - p[i]);
      nxt[j + 1] += dist[j] * p[i];
    }
    dist.swap(nxt);
  }
  double t = 0.0;
  for (size_t j = k; j < dist.size(); ++j) t += dist[j];
  *out = t;
  return SAS_OK;
}

int sas_param_dx_scan(double nu, double nu_th, const double* a, uint32_t n_epochs, const double* dx, uint32_t n_dx,
                      double dv, double dt, double omega, double n_false, double* e_signal, double* e_noise,
                      uint32_t* n_min) {
  if ((n_epochs && !a) || (n_dx && (!dx || !e_signal || !e_noise || !n_min)))
    return set_error(SAS_ERR_ARG, "null argument");
  if (!std::isfinite(nu) || !std::isfinite(nu_th) || !finite_pos(dv) || !finite_pos(dt) || !finite_pos(omega) ||
      !(n_false > 0))
    return set_error(SAS_ERR_ARG, "need finite S/N values and dv, dt, omega, n_false > 0");
  for (uint32_t i = 0; i < n_epochs; ++i)
    if (!finite_pos(a[i])) return set_error(SAS_ERR_ARG, "PSF widths must be > 0");
  for (uint32_t j = 0; j < n_dx; ++j)
    if (!finite_pos(dx[j])) return set_error(SAS_ERR_ARG, "bin sizes must be > 0");
  const double lam1 = peaks_above(nu_th, 1.0);
  for (uint32_t j = 0; j < n_dx; ++j) {
    double en = 0.0;
    for (uint32_t i = 0; i < n_epochs; ++i) en += lam1 * (dx[j] / a[i]) * (dx[j] / a[i]);
    if (!(en <= 1e7)) return set_error(SAS_ERR_RANGE, "noise rate above 1e7 for a bin size");
  }
  for (uint32_t j = 0; j < n_dx; ++j) {
    double es = 0.0, en = 0.0;
    for (uint32_t i = 0; i < n_epochs; ++i) {
      es += p_signal(nu, nu_th, a[i], dx[j]);
      en += lam1 * (dx[j] / a[i]) * (dx[j] / a[i]);
    }
    const double nv = (dt * dv / dx[j]) * (dt * dv / dx[j]);
    const double ns = nv * omega / (dx[j] * dx[j]);
    e_signal[j] = es;
    e_noise[j] = en;
    n_min[j] = choose_n_min(en, n_false / ns);
  }
  return SAS_OK;
}

}  // extern "C"
