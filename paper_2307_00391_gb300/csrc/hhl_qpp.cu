// Host part of the QPP nonlinear transform (App. D): sum_k z_k |k> -> ~ sum_k z_k^2 |k> by phase
// estimation of an amplitude-estimation iterate (QADC), a clock-controlled rotation and the
// inverse (QDAC), run as a UNITARY plan on the HHL kernels. These calls build, in FP64 on the
// host, what that plan is made from: the iterate Q, the rotation table, the start state, and
// the projection of the postselected vector that reads the squared amplitudes.
//
// Registers (system index): amplitude-estimation form, data k (low a bits) and address s
// (high a bits), dimension n^2 (n = 2^a); swap-test form (the STEPS 1-5 as printed), per
// address s the data register ua, a clone a1 of the address and the swap-test qubit a2,
// index ua + n a1 + n^2 a2 + 2 n^2 s, dimension 2 n^3.
#include <math.h>
#include <string.h>

#include <vector>

#include "hhl_common.cuh"

namespace hhl {
namespace {

constexpr double kPiQ = 3.14159265358979323846;

// U_V: the Householder reflection I - 2 w w^T / (w^T w), w = e_0 - z, which takes |0> to |z>
// (the identity when z = e_0). Row-major n x n.
std::vector<double> householder(const double* z, int n) {
  std::vector<double> w(n), u((size_t)n * n, 0.0);
  double ww = 0.0;
  for (int i = 0; i < n; ++i) {
    w[i] = (i == 0 ? 1.0 : 0.0) - z[i];
    ww += w[i] * w[i];
  }
  for (int i = 0; i < n; ++i) u[(size_t)i * n + i] = 1.0;
  if (ww < 1e-300) return u;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) u[(size_t)i * n + j] -= 2.0 * w[i] * w[j] / ww;
  return u;
}

// c = a b (row-major, m x m)
std::vector<double> matmul(const std::vector<double>& a, const std::vector<double>& b, int m) {
  std::vector<double> c((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < m; ++l) {
      const double x = a[(size_t)i * m + l];
      if (x == 0.0) continue;
      for (int j = 0; j < m; ++j) c[(size_t)i * m + j] += x * b[(size_t)l * m + j];
    }
  return c;
}

std::vector<double> transpose(const std::vector<double>& a, int m) {
  std::vector<double> t((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) t[(size_t)j * m + i] = a[(size_t)i * m + j];
  return t;
}

bool check_zeta(const double* zeta, int a_bits, int max_bits) {
  return zeta != nullptr && a_bits >= 1 && a_bits <= max_bits;
}

}  // namespace
}  // namespace hhl

extern "C" {

hhl_status hhl_qpp_iterate(const double* zeta, int32_t a_bits, int32_t form, double* q_out) {
  using namespace hhl;
  if (q_out == nullptr || !check_zeta(zeta, a_bits, form == 0 ? 4 : 2) || (form != 0 && form != 1))
    return fail(HHL_ERR_INVALID_ARG, "need zeta, q_out, form 0 (1 <= a_bits <= 4) or 1 (1 <= a_bits <= 2)");
  const int n = 1 << a_bits;
  const std::vector<double> uv = householder(zeta, n);
  if (form == 0) {
    // block k = -U_V S_0 U_V^T S_k on the data register (S_j flips the sign of |j>)
    const int dim = n * n;
    memset(q_out, 0, sizeof(double) * (size_t)dim * dim);
    std::vector<double> s0((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) s0[(size_t)i * n + i] = i == 0 ? -1.0 : 1.0;
    std::vector<double> core = matmul(matmul(uv, s0, n), transpose(uv, n), n);
    for (double& x : core) x = -x;
    for (int k = 0; k < n; ++k)
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          q_out[(size_t)(k * n + i) * dim + (k * n + j)] = core[(size_t)i * n + j] * (j == k ? -1.0 : 1.0);
    return HHL_OK;
  }
  // swap-test form: block s = -A S_s A^T S_good on [ua | a1 | a2], A = (H on a2)(SWAP(ua, a1)
  // controlled by a2)(H on a2)(U_V on ua), S_good = -Z on a2, S_s the flip of |0>_ua |s>_a1 |0>_a2
  const int nn = n * n, m = 2 * nn, dim = n * m;
  std::vector<double> amat((size_t)m * m, 0.0);
  // (U_V on ua): index i + n j + nn b -> sum_i' U_V[i'][i]
  std::vector<double> uvr((size_t)m * m, 0.0);
  for (int b = 0; b < 2; ++b)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        for (int i2 = 0; i2 < n; ++i2) uvr[(size_t)(b * nn + j * n + i2) * m + (b * nn + j * n + i)] = uv[(size_t)i2 * n + i];
  std::vector<double> h2((size_t)m * m, 0.0), cs((size_t)m * m, 0.0);
  const double r = 1.0 / sqrt(2.0);
  for (int x = 0; x < nn; ++x) {
    h2[(size_t)x * m + x] = r;
    h2[(size_t)x * m + nn + x] = r;
    h2[(size_t)(nn + x) * m + x] = r;
    h2[(size_t)(nn + x) * m + nn + x] = -r;
    cs[(size_t)x * m + x] = 1.0;                                       // a2 = 0: identity
    const int i = x % n, j = x / n;
    cs[(size_t)(nn + i * n + j) * m + (nn + x)] = 1.0;                 // a2 = 1: |i>|j> -> |j>|i>
  }
  amat = matmul(matmul(matmul(h2, cs, m), h2, m), uvr, m);
  const std::vector<double> at = transpose(amat, m);
  memset(q_out, 0, sizeof(double) * (size_t)dim * dim);
  for (int s = 0; s < n; ++s) {
    std::vector<double> ss((size_t)m * m, 0.0), sg((size_t)m * m, 0.0);
    for (int x = 0; x < m; ++x) {
      ss[(size_t)x * m + x] = x == n * s ? -1.0 : 1.0;
      sg[(size_t)x * m + x] = x < nn ? -1.0 : 1.0;
    }
    const std::vector<double> blk = matmul(matmul(matmul(amat, ss, m), at, m), sg, m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) q_out[(size_t)(s * m + i) * dim + (s * m + j)] = -blk[(size_t)i * m + j];
  }
  return HHL_OK;
}

hhl_status hhl_qpp_rotation_table(int32_t n_clock, double c, int32_t form, double* theta_out) {
  using namespace hhl;
  if (theta_out == nullptr || n_clock < 1 || n_clock > 16 || (form != 0 && form != 1) || !(fabs(c) <= 1.0))
    return fail(HHL_ERR_INVALID_ARG, "need theta_out, 1 <= n_clock <= 16, form 0 or 1, |c| <= 1");
  const int64_t R = 1LL << n_clock;
  for (int64_t y = 0; y < R; ++y) {
    const double s = sin(kPiQ * (double)y / (double)R);
    // amplitude-estimation form: sin^2(pi y / 2^r) = z^2; swap-test form: 2 sin^2 - 1 = z^2
    const double z2 = form == 0 ? s * s : 2.0 * s * s - 1.0;
    theta_out[y] = 2.0 * asin(c * z2);
  }
  return HHL_OK;
}

hhl_status hhl_qpp_start_state(const double* zeta, int32_t a_bits, int32_t form, double* b_out) {
  using namespace hhl;
  if (b_out == nullptr || !check_zeta(zeta, a_bits, form == 0 ? 4 : 2) || (form != 0 && form != 1))
    return fail(HHL_ERR_INVALID_ARG, "need zeta, b_out, form 0 (1 <= a_bits <= 4) or 1 (1 <= a_bits <= 2)");
  const int n = 1 << a_bits;
  if (form == 0) {  // uniform address (x) |zeta>
    for (int s = 0; s < n; ++s)
      for (int k = 0; k < n; ++k) b_out[s * n + k] = zeta[k] / sqrt((double)n);
    return HHL_OK;
  }
  // STEPS 1-3: (z_i [j = s] +- [i = s] z_j) / (2 sqrt n) at ua = i, a1 = j, address s (+ for a2 = 0)
  const int nn = n * n;
  const double w = 1.0 / (2.0 * sqrt((double)n));
  for (int s = 0; s < n; ++s)
    for (int b = 0; b < 2; ++b)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const double sym = (j == s ? zeta[i] : 0.0), asy = (i == s ? zeta[j] : 0.0);
          b_out[s * 2 * nn + b * nn + j * n + i] = w * (b == 0 ? sym + asy : sym - asy);
        }
  return HHL_OK;
}

hhl_status hhl_qpp_project(const double* v, const double* b_start, int32_t a_bits, int32_t form, double* squares_out) {
  using namespace hhl;
  if (v == nullptr || b_start == nullptr || squares_out == nullptr || a_bits < 1 || a_bits > (form == 0 ? 4 : 2) ||
      (form != 0 && form != 1))
    return fail(HHL_ERR_INVALID_ARG, "need v, b_start, squares_out, form 0 (1 <= a_bits <= 4) or 1 (1 <= a_bits <= 2)");
  const int n = 1 << a_bits;
  const int block = form == 0 ? n : 2 * n * n;  // amplitudes per address
  const double rn = sqrt((double)n);
  for (int s = 0; s < n; ++s) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < block; ++k) {
      const double st = b_start[s * block + k] * rn;  // the address block's start state, normalised
      re += st * v[2 * (s * block + k)];
      im += st * v[2 * (s * block + k) + 1];
    }
    squares_out[2 * s] = re;
    squares_out[2 * s + 1] = im;
  }
  return HHL_OK;
}

}  // extern "C"
