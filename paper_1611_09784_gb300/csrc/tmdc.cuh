// tmdc.cuh - the TMDC-shaped 11-orbital model (the MoS2 example of Sec. 3.1,
// with the chalcogen-pair vacancies of Sec. 3.2) on an N x N supercell.
//
// Honeycomb lattice a1 = a(1,0), a2 = a(1/2, sqrt3/2): a metal atom with 5 d
// orbitals (q = 0..4) on the A site and a chalcogen pair with 6 p orbitals
// (q = 5..10) on the B site tau_X = (a1 + a2)/3.  Orbital o = 11 c + q, cell
// c = i + N j.  Parameters (real, table P of kTmdcParams doubles):
//   eps[11]        on-site energies                          P[0 .. 10]
//   T1[3][5][6]    metal -> pair, bond b along R_b            P[11 ..]
//                  (R_0 = tau_X, R_1 = tau_X - a1, R_2 = tau_X - a2)
//   T2M[3][5][5]   metal -> metal along +delta_d               P[101 ..]
//   T2X[3][6][6]   pair -> pair along +delta_d                 P[176 ..]
//                  (delta_0 = a1, delta_1 = a2, delta_2 = a2 - a1)
// The pair -> metal hop is T1^T with the conjugate phase, the hop along
// -delta_d is T2[d]^T with the conjugate phase, so H(k) is Hermitian.  Every
// phase is exp(i k . R) of the true bond vector (atomic gauge, eq. (3.2b)),
// reduced as an exact integer fraction before one sincospi call.
#pragma once

#include "graphene.cuh"

namespace idos {

constexpr int kTmdcOrb = 11, kTmdcM = 5, kTmdcX = 6;
constexpr int kTmdcEps = 0, kTmdcT1 = 11, kTmdcT2M = 101, kTmdcT2X = 176, kTmdcParams = 284;

// exp(i k . delta_d) on the K x K grid: k . delta / (2 pi) = (U1 c1 + U2 c2) / (2 N K)
// with U = 2 i - K + 1 and delta_d = c1 a1 + c2 a2.
__device__ __forceinline__ double2 tmdc_second_phase(int N, int K, int kidx, int d) {
  const int i1 = kidx % K, i2 = kidx / K;
  const long long U1 = 2 * i1 - K + 1, U2 = 2 * i2 - K + 1;
  const long long c1 = d == 0 ? 1 : (d == 1 ? 0 : -1), c2 = d == 0 ? 0 : 1;
  const long long D = 2LL * N * K;
  long long num = (U1 * c1 + U2 * c2) % D;
  if (num < 0) num += D;
  double s, c;
  sincospi((double)num / (double)(N * K), &s, &c);   // angle = 2 pi num / D
  return make_double2(c, s);
}

__device__ __forceinline__ int tmdc_cell(int N, int i, int j) {
  i %= N;
  j %= N;
  if (i < 0) i += N;
  if (j < 0) j += N;
  return i + N * j;
}

// Row of orbital o of H(k): add(o', value) for every hop o -> o' (on-site
// included; hops into a removed pair are skipped, removed(cell) tells which
// pairs are gone).  Hops that land on the same o' (small N) accumulate.
template <typename Removed, typename Add>
__device__ __forceinline__ void tmdc_row(int N, int K, int kidx, int o, const double* __restrict__ P,
                                         Removed removed, Add add) {
  const int c = o / kTmdcOrb, q = o % kTmdcOrb;
  const int i = c % N, j = c / N;
  add(o, make_double2(P[kTmdcEps + q], 0.0));
  if (q < kTmdcM) {
    const int mu = q;
    for (int b = 0; b < 3; ++b) {
      const int cb = tmdc_cell(N, i - (b == 1), j - (b == 2));
      if (removed(cb)) continue;
      const double2 ph = graphene_phase(N, K, kidx, b);
      for (int nu = 0; nu < kTmdcX; ++nu) {
        const double t = P[kTmdcT1 + 30 * b + 6 * mu + nu];
        add(kTmdcOrb * cb + kTmdcM + nu, make_double2(t * ph.x, t * ph.y));
      }
    }
    for (int d = 0; d < 3; ++d) {
      const double2 ph = tmdc_second_phase(N, K, kidx, d);
      const int di = d == 0 ? 1 : (d == 1 ? 0 : -1), dj = d == 0 ? 0 : 1;
      const int cf = tmdc_cell(N, i + di, j + dj), cr = tmdc_cell(N, i - di, j - dj);
      for (int m2 = 0; m2 < kTmdcM; ++m2) {
        const double tf = P[kTmdcT2M + 25 * d + 5 * mu + m2];   // T2M[d][mu][m2] along +delta_d
        const double tr = P[kTmdcT2M + 25 * d + 5 * m2 + mu];   // T2M[d]^T along -delta_d
        add(kTmdcOrb * cf + m2, make_double2(tf * ph.x, tf * ph.y));
        add(kTmdcOrb * cr + m2, make_double2(tr * ph.x, -tr * ph.y));
      }
    }
  } else {
    const int nu = q - kTmdcM;
    for (int b = 0; b < 3; ++b) {
      const int cm = tmdc_cell(N, i + (b == 1), j + (b == 2));   // the metal whose bond b ends here
      const double2 ph = graphene_phase(N, K, kidx, b);
      for (int mu = 0; mu < kTmdcM; ++mu) {
        const double t = P[kTmdcT1 + 30 * b + 6 * mu + nu];
        add(kTmdcOrb * cm + mu, make_double2(t * ph.x, -t * ph.y));
      }
    }
    for (int d = 0; d < 3; ++d) {
      const double2 ph = tmdc_second_phase(N, K, kidx, d);
      const int di = d == 0 ? 1 : (d == 1 ? 0 : -1), dj = d == 0 ? 0 : 1;
      const int cf = tmdc_cell(N, i + di, j + dj), cr = tmdc_cell(N, i - di, j - dj);
      const bool gf = removed(cf), gr = removed(cr);
      for (int n2 = 0; n2 < kTmdcX; ++n2) {
        const double tf = P[kTmdcT2X + 36 * d + 6 * nu + n2];
        const double tr = P[kTmdcT2X + 36 * d + 6 * n2 + nu];
        if (!gf) add(kTmdcOrb * cf + kTmdcM + n2, make_double2(tf * ph.x, tf * ph.y));
        if (!gr) add(kTmdcOrb * cr + kTmdcM + n2, make_double2(tr * ph.x, -tr * ph.y));
      }
    }
  }
}

}  // namespace idos
