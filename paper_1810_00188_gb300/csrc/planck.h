// Band blackbody intensity for mcrt_set_kdist's computed tables (host code).
//
// Section 2.2 tabulates, for each narrow band, the blackbody intensity at the
// band centre times the band width: dnu 2 h c^2 nu^3 / (exp(h c nu / (k T)) - 1)
// with wavenumbers in 1/m (the arguments are in 1/cm) and the exact SI values of
// h, c and k.  T <= 0 gives 0; where exp overflows (h c nu / (k T) > 709.78) the
// quotient is 0 as well.
#pragma once

#include <cmath>

namespace mcrt {

inline double planck_band(double nu_c_cm, double dnu_cm, double T) {
  if (!(T > 0.0)) return 0.0;
  const double h = 6.62607015e-34, c = 299792458.0, k = 1.380649e-23;
  const double nu = 100.0 * nu_c_cm, dnu = 100.0 * dnu_cm;
  return dnu * 2.0 * h * (c * c) * std::pow(nu, 3.0) / std::expm1(h * c * nu / (k * T));
}

}  // namespace mcrt
