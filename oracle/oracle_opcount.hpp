// Test infrastructure only: an operation-counting scalar for the FP64 oracle. Every add, subtract,
// multiply, divide, negate-free arithmetic op, sqrt, sin and cos performed on it increments a
// thread-local counter; comparisons are not counted. Running the oracle's step with this scalar
// gives the algorithmic floating-point operation count of the method on an actual trajectory.
// Pinned (tests/test_oracle_opcount.py): each counted operation type counts once and the free ones
// not at all, helper routines and the Cholesky factor / solve match hand-derived closed forms, and
// the solve's cost per position and velocity iteration matches its hand count on the whole step.
#pragma once
#include <cmath>
#include <cstdint>

namespace orc {

struct OpCount {
  double v;
  static uint64_t& counter() {
    static thread_local uint64_t n = 0;
    return n;
  }
  static void reset() { counter() = 0; }
  static uint64_t count() { return counter(); }
  OpCount() : v(0.0) {}
  OpCount(double x) : v(x) {}  // NOLINT: implicit by design (constants)
  friend OpCount operator+(const OpCount& a, const OpCount& b) { ++counter(); return OpCount(a.v + b.v); }
  friend OpCount operator-(const OpCount& a, const OpCount& b) { ++counter(); return OpCount(a.v - b.v); }
  friend OpCount operator*(const OpCount& a, const OpCount& b) { ++counter(); return OpCount(a.v * b.v); }
  friend OpCount operator/(const OpCount& a, const OpCount& b) { ++counter(); return OpCount(a.v / b.v); }
  OpCount operator-() const { return OpCount(-v); }
  friend bool operator<(const OpCount& a, const OpCount& b) { return a.v < b.v; }
  friend bool operator==(const OpCount& a, const OpCount& b) { return a.v == b.v; }
};
inline OpCount sqrt(const OpCount& a) { ++OpCount::counter(); return OpCount(std::sqrt(a.v)); }
inline OpCount sin(const OpCount& a) { ++OpCount::counter(); return OpCount(std::sin(a.v)); }
inline OpCount cos(const OpCount& a) { ++OpCount::counter(); return OpCount(std::cos(a.v)); }
inline OpCount fabs(const OpCount& a) { return OpCount(std::fabs(a.v)); }  // a sign flip, not counted
inline OpCount atan2(const OpCount& y, const OpCount& x) { ++OpCount::counter(); return OpCount(std::atan2(y.v, x.v)); }
inline double val(const OpCount& a) { return a.v; }

}  // namespace orc
