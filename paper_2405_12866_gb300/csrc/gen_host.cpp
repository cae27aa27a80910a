// The method's random draws (host): training states and initial gates.
//
// Philox4x32-10 follows its published definition (Salmon, Moraes, Dror,
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
// two 32x32->64 multiplies with the constants 0xD2511F53 / 0xCD9E8D57 and a
// Weyl key schedule 0x9E3779B9 / 0xBB67AE85.  One block (counter = index,
// stream) gives two 53-bit uniforms and, by Box-Muller, one standard complex
// normal.  The Q factor (positive real R diagonal) of a complex Gaussian
// matrix is Haar distributed (Mezzadri 2007); the training states are such
// columns, as the paper's Appendix A describes them.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

namespace qfs {

namespace {
inline void philox_round(uint32_t c[4], uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0], n1 = lo1, n2 = hi0 ^ c[3] ^ k[1], n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  k[0] += 0x9E3779B9u;
  k[1] += 0xBB67AE85u;
}

inline double u53(uint32_t hi, uint32_t lo) {
  return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}
}  // namespace

void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) philox_round(c, k);
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

std::complex<double> complex_normal(uint64_t seed, uint32_t stream, uint64_t index) {
  const uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32), stream, 0u};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  philox4x32_10(ctr, key, x);
  const double a = u53(x[0], x[1]), b = u53(x[2], x[3]);
  const double r = std::sqrt(-2.0 * std::log(a)) * std::sqrt(0.5);
  const double t = 2.0 * 3.14159265358979323846 * b;
  return {r * std::cos(t), r * std::sin(t)};
}

// Orthonormalise the columns of a (rows x cols, row-major) in place by
// modified Gram-Schmidt applied twice; the implied R has a positive real
// diagonal, so the result is the unique such Q.
void positive_q(std::complex<double>* a, int rows, int cols) {
  for (int j = 0; j < cols; ++j) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = 0; i < j; ++i) {
        std::complex<double> d = 0.0;
        for (int r = 0; r < rows; ++r) d += std::conj(a[(size_t)r * cols + i]) * a[(size_t)r * cols + j];
        for (int r = 0; r < rows; ++r) a[(size_t)r * cols + j] -= d * a[(size_t)r * cols + i];
      }
    }
    double nn = 0.0;
    for (int r = 0; r < rows; ++r) nn += std::norm(a[(size_t)r * cols + j]);
    const double inv = 1.0 / std::sqrt(nn);
    for (int r = 0; r < rows; ++r) a[(size_t)r * cols + j] *= inv;
  }
}

void generate_states(uint64_t seed, uint32_t stream, int n, int M, std::complex<double>* out) {
  const size_t N = (size_t)1 << n;
  for (size_t i = 0; i < N * (size_t)M; ++i) out[i] = complex_normal(seed, stream, i);
  positive_q(out, (int)N, M);
}

// M distinct computational-basis states, uniform without replacement: a
// partial Fisher-Yates shuffle of 0..N-1 in which step j swaps position j
// with j + floor(w_j (N - j) / 2^32), w_j = word 0 of Philox block j of
// (seed, stream).  Column j of out (N x M, row-major) is e_{perm[j]}.
void generate_basis_states(uint64_t seed, uint32_t stream, int n, int M, std::complex<double>* out) {
  const size_t N = (size_t)1 << n;
  std::vector<uint32_t> perm(N);
  for (size_t i = 0; i < N; ++i) perm[i] = (uint32_t)i;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int j = 0; j < M; ++j) {
    const uint32_t ctr[4] = {(uint32_t)j, 0u, stream, 0u};
    uint32_t x[4];
    philox4x32_10(ctr, key, x);
    const size_t r = (size_t)j + (size_t)(((uint64_t)x[0] * (uint64_t)(N - (size_t)j)) >> 32);
    const uint32_t t = perm[j];
    perm[j] = perm[r];
    perm[r] = t;
  }
  std::fill(out, out + N * (size_t)M, std::complex<double>(0.0, 0.0));
  for (int j = 0; j < M; ++j) out[(size_t)perm[j] * M + j] = 1.0;
}

// States of distribution kind (0: Haar, 1: computational basis).
void draw_states(int kind, uint64_t seed, uint32_t stream, int n, int M, std::complex<double>* out) {
  if (kind == 1) generate_basis_states(seed, stream, n, M, out);
  else generate_states(seed, stream, n, M, out);
}

void generate_samples(uint64_t seed, int n, int M, std::complex<double>* out) {
  generate_states(seed, 1u, n, M, out);
}

void generate_gates(uint64_t seed, int count, std::complex<double>* out) {
  for (int g = 0; g < count; ++g) {
    std::complex<double>* q = out + (size_t)16 * g;
    for (int e = 0; e < 16; ++e) q[e] = complex_normal(seed, 2u, (uint64_t)16 * g + e);
    positive_q(q, 4, 4);
  }
}

}  // namespace qfs
