// rpy_dev.h -- RPY pair coefficients (Sec. 3 Eqs. (8)-(9)), shared by the
// assembly of D and the formation of the rod-coupling matrix from positions.
#pragma once

namespace bd {

// Coefficients of D_ij = cI * I + cRR * R R^T for separation R (|R|^2 = R2).
// Eq. (8) for R >= 2a, Eq. (9) for R < 2a, the overlap limit (h*/a) I at R = 0.
template <typename C>
__device__ __forceinline__ void rpy_coeffs(C R2, C hstar, C a, C& cI, C& cRR) {
  const C Rn = sqrt(R2);
  if (hstar == C(0)) {
    cI = C(0);
    cRR = C(0);
  } else if (Rn >= C(2) * a) {
    const C pref = C(0.75) * hstar / Rn;
    const C a2R2 = a * a / R2;
    cI = pref * (C(1) + C(2) / C(3) * a2R2);
    cRR = pref * (C(1) - C(2) * a2R2) / R2;
  } else {
    const C pref = C(0.375) * hstar / a;
    cI = pref * (C(8) / C(3) - C(0.75) * Rn / a);
    cRR = (Rn > C(0)) ? pref * (C(0.25) / a) / Rn : C(0);
  }
}

}  // namespace bd
