// Host-side check of the fixed-point conversions of the deterministic grid sums
// (fix_round, ll_to_float_rn in mpm_common.cuh, compiled here as host code) against the C
// library's correctly rounded conversions: float -> nearest int64 (ties to even) for
// |c| <= 2^55, and int64 -> nearest float (ties to even).  Prints the number of mismatches.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_1910_00935_gb300/csrc/mpm_common.cuh"

int main() {
  std::mt19937_64 g(3);
  long long bad_round = 0, bad_float = 0, n = 0;
  // float -> int64: random magnitudes over [2^-4, 2^55], both signs, plus ties and edges
  std::uniform_real_distribution<double> ue(-4.0, 55.0);
  for (int t = 0; t < 2000000; ++t) {
    float c = (float)std::ldexp(1.0 + (g() >> 11) * 0x1.0p-53, (int)std::floor(ue(g)));
    if (c > 0x1.0p55f) c = 0x1.0p55f;
    if (t & 1) c = -c;
    if (t % 97 == 0) c = (float)((long long)(g() % 2000001) - 1000000) + 0.5f;  // ties
    const long long ref = llrintf(c);
    if (mpm::fix_round(c) != ref) ++bad_round;
    ++n;
  }
  // int64 -> float: random 64-bit values over all magnitudes, plus halfway cases
  for (int t = 0; t < 2000000; ++t) {
    const int bits = 1 + (int)(g() % 63);
    long long a = (long long)(g() >> (64 - bits));
    if (t % 5 == 0 && bits > 25) a = (a | (1ll << (bits - 25))) & ~((1ll << (bits - 25)) - 1);  // a tie
    if (t & 1) a = -a;
    const float ref = (float)a;
    if (mpm::ll_to_float_rn(a) != ref) ++bad_float;
  }
  std::printf("%lld %lld %lld\n", n, bad_round, bad_float);
  return 0;
}
