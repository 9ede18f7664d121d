// Host-side (FP64) plan construction: kernels, u-grid, C matrices, Jacobi
// eigen-decomposition, truncation, cell tables and FFT twiddles.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace sigw {

static const double kSqrt3 = 1.7320508075688772935;
static const double kPi = 3.14159265358979323846;

// Eq. eq_kernels: I_s = 27 pi (u^2+v^2-3)^2 / (32 u^3 v^3) Theta(u+v-sqrt3)
double kernel_Is(double u, double v) {
  if (!(u + v - kSqrt3 > 0.0)) return 0.0;
  const double a = u * u + v * v - 3.0;
  return 27.0 * kPi * a * a / (32.0 * u * u * u * v * v * v);
}

// Eq. eq_kernels: I_c = 27 (u^2+v^2-3) / (32 u^3 v^3) (-4uv + (u^2+v^2-3) ln|(3-(u+v)^2)/(3-(u-v)^2)|)
double kernel_Ic(double u, double v) {
  const double a = u * u + v * v - 3.0;
  const double s = u + v, d = u - v;
  const double lg = std::log(std::fabs((3.0 - s * s) / (3.0 - d * d)));
  return 27.0 * a / (32.0 * u * u * u * v * v * v) * (-4.0 * u * v + a * lg);
}

// Integral of the grid density rho(u) = 1 + Ap exp(-(u-up)^2/(2 sp^2)) from umin to u (closed form).
static double cum_density(double u, const DecompParams& p) {
  const double s2 = std::sqrt(2.0) * p.sigp;
  return (u - p.umin) + p.Ap * p.sigp * std::sqrt(kPi / 2.0) *
                            (std::erf((u - p.upiv) / s2) - std::erf((p.umin - p.upiv) / s2));
}

void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += a(i, i) * a(i, i);
      for (int j = i + 1; j < n; ++j) off += a(i, j) * a(i, j);
    }
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = a(p, q);
        if (apq == 0.0) continue;
        const double app = a(p, p), aqq = a(q, q);
        // rotation angle annihilating a(p,q): tan(2 theta) = 2 apq / (aqq - app)
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        a(p, q) = 0.0;
        a(q, p) = 0.0;
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a(i, i);
}

bool build_decomposition(const DecompParams& p, Decomposition* out, std::string* err) {
  if (p.n_modes < 2 || p.n_modes > 4096 || p.n_alpha < 1 || p.n_alpha > p.n_modes || !(p.umin > 0) ||
      !(p.umax > p.umin) || !(p.sigp > 0) || !(p.Ap >= 0)) {
    if (err) *err = "invalid decomposition parameters";
    return false;
  }
  const int n = p.n_modes;
  Decomposition d;
  d.p = p;
  // 1. edges e_n = u(n), n = 0..n_modes: equal integrated density between edges (bisection)
  d.edges.resize(n + 1);
  const double Rmax = cum_density(p.umax, p);
  d.edges[0] = p.umin;
  d.edges[n] = p.umax;
  for (int k = 1; k < n; ++k) {
    const double target = k * Rmax / n;
    double lo = p.umin, hi = p.umax;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (cum_density(mid, p) < target) lo = mid; else hi = mid;
      if (hi - lo <= 1e-15 * std::max(1.0, std::fabs(mid))) break;
    }
    d.edges[k] = 0.5 * (lo + hi);
  }
  d.centres.resize(n);
  d.widths.resize(n);
  for (int i = 0; i < n; ++i) {
    d.centres[i] = 0.5 * (d.edges[i] + d.edges[i + 1]);
    d.widths[i] = d.edges[i + 1] - d.edges[i];
  }
  for (int m = 0; m < 2; ++m) {
    // 2. C_ij = sqrt(L_i L_j) I(u_i, u_j) where (u_i, u_j, 1) can form a triangle
    std::vector<double> C((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) {
        const double ui = d.centres[i], uj = d.centres[j];
        if (std::fabs(ui - uj) <= 1.0 && ui + uj >= 1.0) {
          const double I = (m == 0) ? kernel_Is(ui, uj) : kernel_Ic(ui, uj);
          C[(size_t)i * n + j] = std::sqrt(d.widths[i] * d.widths[j]) * I;
        }
      }
    }
    // symmetrise exactly (I is symmetric; guard against last-bit asymmetry of pow/log)
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        const double s = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
        C[(size_t)i * n + j] = C[(size_t)j * n + i] = s;
      }
    // 3. eigen-decomposition and truncation by |sigma| (ties by index)
    std::vector<double> w, V;
    jacobi_eigen(n, C, w, V);
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(w[a]) > std::fabs(w[b]); });
    KernelTerms& t = d.terms[m];
    t.sigma.resize(p.n_alpha);
    t.phi.assign((size_t)p.n_alpha * n, 0.0);
    for (int a = 0; a < p.n_alpha; ++a) {
      const int k = order[a];
      t.sigma[a] = w[k];
      for (int i = 0; i < n; ++i) t.phi[(size_t)a * n + i] = V[(size_t)i * n + k] / std::sqrt(d.widths[i]);
    }
  }
  *out = std::move(d);
  return true;
}

void build_cell_lut(const std::vector<double>& edges, int n_c, int msq_max, int16_t* lut) {
  const int n_modes = (int)edges.size() - 1;
  std::vector<double> thr(edges.size());
  for (size_t i = 0; i < edges.size(); ++i) thr[i] = (edges[i] * n_c) * (edges[i] * n_c);
  int k = 0;  // number of thresholds <= msq (monotone in msq)
  for (int msq = 0; msq <= msq_max; ++msq) {
    while (k < (int)thr.size() && thr[k] <= (double)msq) ++k;
    const int cell = k - 1;
    lut[msq] = (int16_t)((k == 0 || k == (int)thr.size()) ? n_modes : cell);
  }
}

void build_twiddles(int n, std::vector<double>& tw) {
  tw.resize(2 * (size_t)n);
  for (int k = 0; k < n; ++k) {
    const double a = -2.0 * kPi * (double)k / (double)n;
    tw[2 * k] = std::cos(a);
    tw[2 * k + 1] = std::sin(a);
  }
}

}  // namespace sigw
