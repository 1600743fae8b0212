// Test infrastructure only: a forward-mode dual number (value, one tangent) for the FP64 oracle.
// Running the oracle's step on it gives the exact directional derivative of the discrete FP64 step
// along the seeded input tangent: each elementary operation carries its derivative by the chain
// rule; comparisons and branches (contact and limit decisions, clamps, the speculative / biased
// target choice) follow the value, so the derivative is that of the step with its constraint and
// active sets held fixed. This is the oracle gradient the adjoint of the CUDA path is checked
// against.
#pragma once
#include <cmath>

namespace orc {

struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}  // NOLINT: implicit by design (constants)
  Dual(double x, double dx) : v(x), d(dx) {}
  friend Dual operator+(const Dual& a, const Dual& b) { return Dual(a.v + b.v, a.d + b.d); }
  friend Dual operator-(const Dual& a, const Dual& b) { return Dual(a.v - b.v, a.d - b.d); }
  friend Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
  friend Dual operator/(const Dual& a, const Dual& b) {
    const double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
  }
  Dual operator-() const { return Dual(-v, -d); }
  friend bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
  friend bool operator==(const Dual& a, const Dual& b) { return a.v == b.v; }
};
inline Dual sqrt(const Dual& a) {
  const double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline Dual sin(const Dual& a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
inline Dual cos(const Dual& a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
inline Dual fabs(const Dual& a) { return a.v < 0.0 ? -a : a; }
inline double val(const Dual& a) { return a.v; }

}  // namespace orc
