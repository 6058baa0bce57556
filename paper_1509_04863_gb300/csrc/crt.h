// Steps 8-9 of Algorithm 1 in closed form (Thm. 4, Chinese remainder).
//
// S_i = {(m_i + l M_i) mod N : 0 <= l < L_i}, L_i = ceil(N / M_i). An
// element of S_i is either "natural" (m_i + l M_i < N, i.e. any v < N with
// v = m_i mod M_i) or the single wrapped member w_i = m_i + (L_i-1) M_i - N,
// present when w_i >= 0. Hence S1 ∩ S2 consists of
//   - the naturals v < N with v = m1 (mod M1), v = m2 (mod M2): the
//     progression m0 + j M1 M2, m0 the CRT solution in [0, M1 M2);
//   - w1 when it lies in S2, and w2 when it lies in S1 (w_i is never
//     congruent to m_i mod M_i, so it is never a natural of S_i).
#pragma once

#include <cstdint>

namespace ftm {

struct CrtSet {
  int64_t m0;      // first natural solution (>= N when there is none)
  int64_t step;    // M1 * M2 (M1 * M2 * M3)
  int64_t nnat;    // number of natural solutions below N
  int64_t w[3];    // wrapped members in the intersection
  int32_t nw;
};

#if defined(__CUDACC__)
#define TM_HD __host__ __device__ __forceinline__
#else
#define TM_HD inline
#endif

// Modular inverse of a mod m (gcd(a, m) = 1, m >= 1), by extended Euclid.
TM_HD int64_t mod_inverse(int64_t a, int64_t m) {
  if (m == 1) return 0;
  int64_t r0 = m, r1 = ((a % m) + m) % m, s0 = 0, s1 = 1;
  while (r1 != 0) {
    const int64_t qq = r0 / r1;
    int64_t tmp = r0 - qq * r1; r0 = r1; r1 = tmp;
    tmp = s0 - qq * s1; s0 = s1; s1 = tmp;
  }
  return ((s0 % m) + m) % m;
}

// With L_i = ceil(N / M_i) given (the device has them in its descriptors).
// 64-bit divisions are long instruction sequences on a GPU: the common cases
// (residues already reduced, one natural solution, wrapped members below
// the other modulus) skip them; the results are those of the plain
// formulas in every case.
TM_HD CrtSet crt_intersect_L(int64_t N, int64_t M1, int64_t M2, int64_t L1, int64_t L2, int64_t inv, int64_t m1,
                             int64_t m2) {
  CrtSet c;
  // m0 = m1 + M1 * k with M1 * k = m2 - m1 (mod M2)
  int64_t d = m2 - m1;
  if (d < 0) d += M2;
  if (d < 0 || d >= M2) d = ((m2 - m1) % M2 + M2) % M2;
  const int64_t k = int64_t(uint64_t(d) * uint64_t(inv) % uint64_t(M2));   // d, inv < M2 < 2^31
  c.m0 = m1 + M1 * k;
  c.step = M1 * M2;
  const int64_t span = N - 1 - c.m0;
  c.nnat = c.m0 < N ? (span < c.step ? 1 : span / c.step + 1) : 0;
  const int64_t w1 = m1 + (L1 - 1) * M1 - N;
  const int64_t w2 = m2 + (L2 - 1) * M2 - N;
  c.nw = 0;
  if (w1 >= 0 && ((w1 < M2 ? w1 : w1 % M2) == m2 || w1 == w2)) c.w[c.nw++] = w1;
  if (w2 >= 0 && w2 != w1 && (w2 < M1 ? w2 : w2 % M1) == m1) c.w[c.nw++] = w2;
  return c;
}

TM_HD CrtSet crt_intersect(int64_t N, int64_t M1, int64_t M2, int64_t inv, int64_t m1, int64_t m2) {
  return crt_intersect_L(N, M1, M2, (N + M1 - 1) / M1, (N + M2 - 1) / M2, inv, m1, m2);
}

// Three moduli (Thm. 4): the naturals solve v = m_i (mod M_i), i = 1..3,
// the progression m0 + j M1 M2 M3 (m0 from the two-modulus solution and
// inv3 = (M1 M2)^{-1} mod M3); a wrapped member w_i joins when it lies in
// the other two sets (congruent to their m_j, or equal to their w_j).
TM_HD CrtSet crt_intersect3(int64_t N, const int64_t (&M)[3], int64_t inv, int64_t inv3, const int64_t (&m)[3]) {
  CrtSet c = crt_intersect(N, M[0], M[1], inv, m[0], m[1]);
  const int64_t M12 = M[0] * M[1];
  const int64_t d = ((m[2] - c.m0) % M[2] + M[2]) % M[2];
  const int64_t k = (d * inv3) % M[2];
  c.m0 = c.m0 + M12 * k;
  c.step = M12 * M[2];
  c.nnat = c.m0 < N ? (N - 1 - c.m0) / c.step + 1 : 0;
  int64_t w[3];
  for (int i = 0; i < 3; ++i) w[i] = m[i] + ((N + M[i] - 1) / M[i] - 1) * M[i] - N;
  c.nw = 0;
  for (int i = 0; i < 3; ++i) {
    if (w[i] < 0) continue;
    bool all = true, dup = false;
    for (int j = 0; j < 3; ++j)
      if (j != i && !(w[i] % M[j] == m[j] || w[i] == w[j])) all = false;
    for (int q = 0; q < c.nw; ++q) dup = dup || c.w[q] == w[i];
    if (all && !dup) c.w[c.nw++] = w[i];
  }
  return c;
}

#undef TM_HD

}  // namespace ftm
