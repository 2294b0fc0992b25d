// Magnitude arithmetic for running error bounds (test infrastructure only).
//
// Evaluating an expression with every operand replaced by its absolute value,
// and every subtraction by an addition, gives for each result the sum of the
// magnitudes of the terms it is built from.  A floating-point evaluation of
// the same expression in unit roundoff u, from inputs each known to a few u,
// is then within (number of roundings on the longest path + input error) * u
// of that magnitude, to first order (running error analysis: Higham, Accuracy
// and Stability of Numerical Algorithms, 2nd ed., Sec. 3.3).
#pragma once

#include <cmath>

struct Mag {
  double v;
  Mag(double x = 0.0) : v(std::fabs(x)) {}
};

inline Mag mag_of(double v) {
  Mag r;
  r.v = v;
  return r;
}
inline Mag operator+(Mag a, Mag b) { return mag_of(a.v + b.v); }
inline Mag operator-(Mag a, Mag b) { return mag_of(a.v + b.v); }
inline Mag operator*(Mag a, Mag b) { return mag_of(a.v * b.v); }
inline Mag operator/(Mag a, Mag b) { return mag_of(a.v / b.v); }
inline Mag operator-(Mag a) { return a; }
inline Mag& operator+=(Mag& a, Mag b) { return a = a + b; }
inline Mag& operator-=(Mag& a, Mag b) { return a = a - b; }
