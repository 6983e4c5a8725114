// stats.cpp -- host statistics of the Section 5 normality procedure:
// normalised deviations of batch values and the Shapiro-Wilk test with
// Royston's approximation (Royston 1992, Stat. Comput. 2:117-119; Algorithm
// AS R94, Appl. Statist. 44:547-551, 1995).  Post-processing of a few
// thousand numbers per call; it runs on the host.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/mc.h"

namespace {

double phi_upper(double z) { return 0.5 * std::erfc(z / std::sqrt(2.0)); }

// Standard normal quantile: rational starting value (Abramowitz & Stegun
// 26.2.23, |error| < 4.5e-4) refined by Halley steps on erfc, which
// converge to full double precision in two or three steps.
double norm_quantile(double p) {
  const bool lower = p < 0.5;
  const double q = lower ? p : 1.0 - p;
  const double t = std::sqrt(-2.0 * std::log(q));
  double x = t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                     (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t);
  x = lower ? -x : x;
  for (int it = 0; it < 4; ++it) {
    const double cdf = 0.5 * std::erfc(-x / std::sqrt(2.0));
    const double pdf = std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI);
    const double e = (cdf - p) / pdf;
    x = x - e / (1.0 + 0.5 * x * e);
  }
  return x;
}

double horner(const double* c, int n, double x) {
  double r = c[n - 1];
  for (int i = n - 2; i >= 0; --i) r = r * x + c[i];
  return r;
}

// W and p for one sample; returns false if n is out of range or the
// sample has no spread.
bool swilk(std::vector<double> x, double* w_out, double* p_out) {
  const int n = (int)x.size();
  if (n < 3 || n > 5000) return false;
  std::sort(x.begin(), x.end());
  double mean = 0.0;
  for (double v : x) mean += v;
  mean /= n;
  double ss = 0.0;
  for (double v : x) ss += (v - mean) * (v - mean);
  if (!(ss > 0.0)) return false;

  const int half = n / 2;
  std::vector<double> a(half);  // weights of the upper half, a[0] = largest
  if (n == 3) {
    a[0] = std::sqrt(0.5);
  } else {
    std::vector<double> m(half);
    double mm = 0.0;
    for (int i = 0; i < half; ++i) {
      m[i] = -norm_quantile(((double)(i + 1) - 0.375) / ((double)n + 0.25));  // m_n, m_{n-1}, ...
      mm += 2.0 * m[i] * m[i];
    }
    const double u = 1.0 / std::sqrt((double)n);
    static const double c1[6] = {0.0, 0.221157, -0.147981, -2.071190, 4.434685, -2.706056};
    static const double c2[6] = {0.0, 0.042981, -0.293762, -1.752461, 5.682633, -3.582633};
    const double rm = std::sqrt(mm);
    a[0] = m[0] / rm + horner(c1, 6, u);
    int first;
    double phi;
    if (n > 5) {
      a[1] = m[1] / rm + horner(c2, 6, u);
      phi = (mm - 2.0 * m[0] * m[0] - 2.0 * m[1] * m[1]) / (1.0 - 2.0 * a[0] * a[0] - 2.0 * a[1] * a[1]);
      first = 2;
    } else {
      phi = (mm - 2.0 * m[0] * m[0]) / (1.0 - 2.0 * a[0] * a[0]);
      first = 1;
    }
    for (int i = first; i < half; ++i) a[i] = m[i] / std::sqrt(phi);
  }
  double b = 0.0;
  for (int i = 0; i < half; ++i) b += a[i] * (x[n - 1 - i] - x[i]);
  double W = b * b / ss;
  if (W > 1.0) W = 1.0;

  double p;
  if (n == 3) {
    if (W < 0.75) W = 0.75;
    p = (6.0 / M_PI) * (std::asin(std::sqrt(W)) - std::asin(std::sqrt(0.75)));
  } else if (n <= 11) {
    const double nn = (double)n;
    const double gamma = 0.459 * nn - 2.273;
    static const double cm[4] = {0.5440, -0.39978, 0.025054, -0.0006714};
    static const double cs[4] = {1.3822, -0.77857, 0.062767, -0.0020322};
    const double mu = horner(cm, 4, nn), sigma = std::exp(horner(cs, 4, nn));
    const double y = std::log1p(-W);
    p = y >= gamma ? 0.0 : phi_upper((-std::log(gamma - y) - mu) / sigma);
  } else {
    const double ln = std::log((double)n);
    static const double cm[4] = {-1.5861, -0.31082, -0.083751, 0.0038915};
    static const double cs[3] = {-0.4803, -0.082676, 0.0030302};
    const double mu = horner(cm, 4, ln), sigma = std::exp(horner(cs, 3, ln));
    p = phi_upper((std::log1p(-W) - mu) / sigma);
  }
  *w_out = W;
  *p_out = p;
  return true;
}

}  // namespace

extern "C" MC_API int mc_normality(const double* h_x, uint32_t n_batches, uint32_t n_points, double* h_z,
                                   double* h_w, double* h_p) {
  if (!h_x || n_batches < 3 || n_batches > 5000) return MC_ERR_ARG;
  int status = MC_OK;
  std::vector<double> col(n_batches);
  for (uint32_t j = 0; j < n_points; ++j) {
    double mean = 0.0;
    for (uint32_t b = 0; b < n_batches; ++b) {
      col[b] = h_x[(size_t)b * n_points + j];
      mean += col[b];
    }
    mean /= n_batches;
    double var = 0.0;
    for (double v : col) var += (v - mean) * (v - mean);
    const double sd = std::sqrt(var / (n_batches - 1));
    if (h_z)
      for (uint32_t b = 0; b < n_batches; ++b) h_z[(size_t)b * n_points + j] = sd > 0.0 ? (col[b] - mean) / sd : 0.0;
    double W = NAN, p = NAN;
    if (!swilk(col, &W, &p)) status = MC_ERR_ARG;
    if (h_w) h_w[j] = W;
    if (h_p) h_p[j] = p;
  }
  return status;
}
