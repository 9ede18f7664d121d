// Host-side (FP64) plan construction for the lattice SIGW library.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace sigw {

struct DecompParams {
  int n_modes = 200, n_alpha = 50;
  double umin = 1e-3, umax = 15.0, upiv = 1.0, sigp = 0.5, Ap = 10.0;
};

// Truncated separable form of one kernel: I(u,v) ~= sum_a sigma[a] phi[a][i(u)] phi[a][i(v)].
struct KernelTerms {
  std::vector<double> sigma;  // n_alpha, |sigma| descending
  std::vector<double> phi;    // n_alpha * n_modes, row-major [a][cell]
};

struct Decomposition {
  DecompParams p;
  std::vector<double> edges;    // n_modes + 1
  std::vector<double> centres;  // n_modes
  std::vector<double> widths;   // n_modes
  KernelTerms terms[2];         // 0: I_s, 1: I_c
};

// Eq. eq_kernels (Theta(0) = 0)
double kernel_Is(double u, double v);
double kernel_Ic(double u, double v);

// Sec. sec_decomposition: grid (Eq. eq_grid_density), C matrix on the triangle strip
// (Eq. eq_C_matrix_discrete), eigen-decomposition (Eq. eq_diagonalization), truncation.
// Returns false (with a message) on invalid parameters.
bool build_decomposition(const DecompParams& p, Decomposition* out, std::string* err);

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major, destroyed).
// On return w[n] holds eigenvalues and V[n*n] (row-major, column k = eigenvector k).
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V);

// Cell of integer |n|^2 = msq for target shell n_c: the i with e_i <= |n|/n_c < e_{i+1}, decided
// on squares ((e_i n_c)^2 <= msq) in FP64; -1 outside [umin, umax).
// Fills lut[msq] for msq = 0..msq_max with the cell index, or n_modes for "outside".
void build_cell_lut(const std::vector<double>& edges, int n_c, int msq_max, int16_t* lut);

// Forward roots tw[k] = exp(-2 pi i k / n), k = 0..n-1, interleaved (re, im), FP64.
void build_twiddles(int n, std::vector<double>& tw);

}  // namespace sigw
