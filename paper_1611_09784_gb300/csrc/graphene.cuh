// graphene.cuh - nearest-neighbour honeycomb model on an N x N supercell
// (Sec. 3.1, eq. (3.2a)-(3.2b)): bond phases and neighbour lists.
//
// Site m = 2(i + N j) + s.  An A site (s = 0) of cell (i, j) bonds to the B
// sites of cells (i, j), (i-1, j), (i, j-1) (indices mod N) along
//   R_0 = tau_B, R_1 = tau_B - a1, R_2 = tau_B - a2,  tau_B = (a1 + a2)/3,
// and a B site bonds back to the A sites of (i, j), (i+1, j), (i, j+1) along
// -R_0, -R_1, -R_2.  With k = (u1 b1 + u2 b2)/N on the Monkhorst-Pack grid,
// u = (2i - K + 1)/(2K) for i = 0..K-1, the phase is exactly
//   k . R_b / (2 pi) = (U1 c1 + U2 c2) / (6 N K),  U = 2i - K + 1,
//   (c1, c2) = 3 R_b in the (a1, a2) basis = (1, 1), (-2, 1), (1, -2),
// so it is reduced as an integer fraction before one sincospi call.
#pragma once

#include "common.cuh"

namespace idos {

__device__ __forceinline__ double2 graphene_phase(int N, int K, int kidx, int b) {
  const int i1 = kidx % K, i2 = kidx / K;
  const long long U1 = 2 * i1 - K + 1, U2 = 2 * i2 - K + 1;
  const long long c1 = (b == 1) ? -2 : 1, c2 = (b == 2) ? -2 : 1;
  const long long D = 6LL * N * K;
  long long num = (U1 * c1 + U2 * c2) % D;
  if (num < 0) num += D;
  double s, c;
  sincospi((double)num / (double)(3LL * N * K), &s, &c);   // angle = 2 pi num / D
  return make_double2(c, s);
}

// float32 variant: the same integer reduction, then one float32 sincospi of
// a fraction in [0, 2) (relative rounding below 2^-23).
__device__ __forceinline__ float2 graphene_phase_f(int N, int K, int kidx, int b) {
  const int i1 = kidx % K, i2 = kidx / K;
  const int U1 = 2 * i1 - K + 1, U2 = 2 * i2 - K + 1;
  const int c1 = (b == 1) ? -2 : 1, c2 = (b == 2) ? -2 : 1;
  const int D = 6 * N * K;
  int num = (U1 * c1 + U2 * c2) % D;
  if (num < 0) num += D;
  float s, c;
  sincospif((float)num / (float)(3 * N * K), &s, &c);
  return make_float2(c, s);
}

// The three neighbours of site m; conj_phase = true for a B site (bond -R_b).
__device__ __forceinline__ void graphene_neighbours(int N, int m, int nb[3], bool& from_B) {
  const int cell = m >> 1, s = m & 1;
  const int i = cell % N, j = cell / N;
  if (s == 0) {
    const int im = (i + N - 1) % N, jm = (j + N - 1) % N;
    nb[0] = 2 * (i + N * j) + 1;
    nb[1] = 2 * (im + N * j) + 1;
    nb[2] = 2 * (i + N * jm) + 1;
    from_B = false;
  } else {
    const int ip = (i + 1) % N, jp = (j + 1) % N;
    nb[0] = 2 * (i + N * j);
    nb[1] = 2 * (ip + N * j);
    nb[2] = 2 * (i + N * jp);
    from_B = true;
  }
}

}  // namespace idos
