// Host-side lattice geometry of the library: the even-odd half-site index and
// the neighbour table.  Plain C++ without CUDA, so that it also compiles on
// its own (the CPU tests check it against the lattice shifts of the oracle).
//
// Directions mu = 0, 1, 2, 3 are x, y, z, t; a site's parity is
// (x + y + z + t) mod 2.  The full-site index is
//   n = ((t * Z + z) * Y + y) * X + x,
// and a site of parity `par` has the half-site index h = n / 2 (X is even, so
// the two sites of an x pair share h and differ in parity):
//   xh = h mod (X / 2),  (y, z, t) from h / (X / 2),  x = 2 xh + ((par + y + z + t) & 1).
#pragma once

namespace dwf {

// nb[d * Vh + h], Vh = X Y Z T / 2: the half-site index (on the other
// parity) of the neighbour n + mu_hat (d = mu < 4) or n - mu_hat (d = 4 + mu)
// of the half site h of parity `par`, periodic in every direction.  Every
// extent must be even and at least 2.
inline void build_neighbour_table(int X, int Y, int Z, int T, int par, int* nb) {
  const long Vh = (long)X * Y * Z * T / 2;
  const int Xh = X / 2;
  const int ext[4] = {X, Y, Z, T};
  for (long h = 0; h < Vh; ++h) {
    long rest = h / Xh;
    const int xh = (int)(h % Xh);
    const int y = (int)(rest % Y);
    rest /= Y;
    const int z = (int)(rest % Z);
    const int t = (int)(rest / Z);
    const int x = 2 * xh + ((par + y + z + t) & 1);
    const int c[4] = {x, y, z, t};
    for (int d = 0; d < 8; ++d) {
      int q[4] = {c[0], c[1], c[2], c[3]};
      const int mu = d & 3;
      q[mu] = (q[mu] + (d < 4 ? 1 : ext[mu] - 1)) % ext[mu];
      const long n = (((long)q[3] * Z + q[2]) * Y + q[1]) * X + q[0];
      nb[(long)d * Vh + h] = (int)(n >> 1);
    }
  }
}

}  // namespace dwf
