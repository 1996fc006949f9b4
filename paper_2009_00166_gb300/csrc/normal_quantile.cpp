// iSAX breakpoints beta_j = Phi^-1(j / card), j = 1..card-1, on the host in FP64.
// Phi^-1 follows M. J. Wichura, "Algorithm AS 241: The Percentage Points of the Normal
// Distribution", Applied Statistics 37(3), 1988 (PPND16, about 1e-16 relative accuracy):
// a rational approximation in (p - 1/2)^2 for central p, and in sqrt(-log(min(p, 1-p)))
// for the tails. Compiled without floating-point contraction so every operation rounds once.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace paris {

static double horner8(const double* c, double r) {
  // c[7] r^7 + ... + c[0], evaluated from the highest coefficient down
  double v = c[7];
  for (int i = 6; i >= 0; --i) v = v * r + c[i];
  return v;
}

double normal_quantile(double p) {
  static const double a[8] = {3.3871328727963666080e+0, 1.3314166789178437745e+2, 1.9715909503065514427e+3,
                              1.3731693765509461125e+4, 4.5921953931549871457e+4, 6.7265770927008700853e+4,
                              3.3430575583588128105e+4, 2.5090809287301226727e+3};
  static const double b[8] = {1.0, 4.2313330701600911252e+1, 6.8718700749205790830e+2,
                              5.3941960214247511077e+3, 2.1213794301586595867e+4, 3.9307895800092710610e+4,
                              2.8729085735721942674e+4, 5.2264952788528545610e+3};
  static const double c[8] = {1.42343711074968357734e+0, 4.63033784615654529590e+0, 5.76949722146069140550e+0,
                              3.64784832476320460504e+0, 1.27045825245236838258e+0, 2.41780725177450611770e-1,
                              2.27238449892691845833e-2, 7.74545014278341407640e-4};
  static const double d[8] = {1.0, 2.05319162663775882187e+0, 1.67638483018380384940e+0,
                              6.89767334985100004550e-1, 1.48103976427480074590e-1, 1.51986665636164571966e-2,
                              5.47593808499534494600e-4, 1.05075007164441684324e-9};
  static const double e[8] = {6.65790464350110377720e+0, 5.46378491116411436990e+0, 1.78482653991729133580e+0,
                              2.96560571828504891230e-1, 2.65321895265761230930e-2, 1.24266094738807843860e-3,
                              2.71155556874348757815e-5, 2.01033439929228813265e-7};
  static const double f[8] = {1.0, 5.99832206555887937690e-1, 1.36929880922735805310e-1,
                              1.48753612908506148525e-2, 7.86869131145613259100e-4, 1.84631831751005468180e-5,
                              1.42151175831644588870e-7, 2.04426310338993978564e-15};
  const double q = p - 0.5;
  if (std::fabs(q) <= 0.425) {
    const double r = 0.180625 - q * q;
    return horner8(a, r) * q / horner8(b, r);
  }
  double r = q <= 0.0 ? p : 1.0 - p;
  r = std::sqrt(-std::log(r));
  double x;
  if (r <= 5.0) {
    r = r - 1.6;
    x = horner8(c, r) / horner8(d, r);
  } else {
    r = r - 5.0;
    x = horner8(e, r) / horner8(f, r);
  }
  return q < 0.0 ? -x : x;
}

std::vector<double> normal_breakpoints(int card) {
  std::vector<double> beta((size_t)card - 1);
  for (int j = 1; j < card; ++j) beta[(size_t)j - 1] = normal_quantile((double)j / (double)card);
  return beta;
}

void breakpoint_tables(const std::vector<double>& beta, std::vector<uint64_t>& keys,
                       std::vector<double>& ext) {
  keys.resize(beta.size());
  ext.resize(beta.size() + 2);
  ext[0] = -INFINITY;
  for (size_t j = 0; j < beta.size(); ++j) {
    double v = beta[j] == 0.0 ? 0.0 : beta[j];
    uint64_t u;
    std::memcpy(&u, &v, sizeof u);
    keys[j] = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
    ext[j + 1] = beta[j];
  }
  ext[beta.size() + 1] = INFINITY;
}

}  // namespace paris
