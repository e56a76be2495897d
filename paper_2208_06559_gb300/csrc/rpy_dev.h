// rpy_dev.h -- RPY pair coefficients (Sec. 3 Eqs. (8)-(9)), for the assembly
// of D and the formation of the rod-coupling matrices from positions.
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

// The same coefficients from one square root and one division (the inverse
// distance; every other quotient becomes a product), for FP64 code where each
// division or square root is a long instruction sequence: the same values up
// to the last bits of the rounding.  inv_a = 1 / a.
template <typename C>
__device__ __forceinline__ void rpy_coeffs_inv(C R2, C hstar, C a, C inv_a, C& cI, C& cRR) {
  if (hstar == C(0)) {
    cI = C(0);
    cRR = C(0);
    return;
  }
  if (R2 > C(0)) {
    const C iR = C(1) / sqrt(R2), iR2 = iR * iR;
    if (R2 >= C(4) * a * a) {  // R >= 2a
      const C pref = C(0.75) * hstar * iR;
      const C a2R2 = a * a * iR2;
      cI = pref * (C(1) + C(2) / C(3) * a2R2);
      cRR = pref * (C(1) - C(2) * a2R2) * iR2;
    } else {
      const C pref = C(0.375) * hstar * inv_a;
      cI = pref * (C(8) / C(3) - C(0.75) * (R2 * iR) * inv_a);
      cRR = pref * (C(0.25) * inv_a) * iR;
    }
  } else {
    cI = C(0.375) * hstar * inv_a * (C(8) / C(3));
    cRR = C(0);
  }
}

// The same coefficients in FP32 from one reciprocal square root (rsqrtf, a
// few ulp) and a precomputed 1 / a instead of a square root and three
// divisions: a relative change of order 1e-7, the size of the FP32 rounding
// itself.  For the formation of K and G from the positions, which evaluates
// one pair per output element and is instruction-bound.
__device__ __forceinline__ void rpy_coeffs_rsqrt(float R2, float hstar, float a, float inv_a, float& cI,
                                                 float& cRR) {
  if (hstar == 0.0f) {
    cI = 0.0f;
    cRR = 0.0f;
    return;
  }
  if (R2 >= 4.0f * a * a) {  // R >= 2a
    const float iR = rsqrtf(R2);
    const float pref = 0.75f * hstar * iR;
    const float a2R2 = a * a * iR * iR;
    cI = pref * (1.0f + (2.0f / 3.0f) * a2R2);
    cRR = pref * (1.0f - 2.0f * a2R2) * iR * iR;
  } else {
    const float pref = 0.375f * hstar * inv_a;
    if (R2 > 0.0f) {
      const float iR = rsqrtf(R2);
      cI = pref * (8.0f / 3.0f - 0.75f * (R2 * iR) * inv_a);
      cRR = pref * (0.25f * inv_a) * iR;
    } else {
      cI = pref * (8.0f / 3.0f);
      cRR = 0.0f;
    }
  }
}

}  // namespace bd
