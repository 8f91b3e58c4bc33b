// Host-side interface of the projected-matrix eigensolve (css_eigen.cu).
#pragma once
#include "css_internal.cuh"

// Fermi-Dirac occupation (1 - tanh((x - mu) / (2 kT))) / 2; beyond |z| = 20 tanh is +-1 in
// FP64, so the value is exactly 0 or 1 there; kT = 0 is the step function (1/2 at x = mu).
__device__ __forceinline__ double css_fermi_dirac(double x, double mu, double kT) {
  if (kT > 0.0) {
    const double z = (x - mu) / (2.0 * kT);
    if (z > 20.0) return 0.0;
    if (z < -20.0) return 1.0;
    return 0.5 * (1.0 - tanh(z));
  }
  return x < mu ? 1.0 : (x > mu ? 0.0 : 0.5);
}

struct EigArgs {
  int32_t n_col = 0, b = 0, m = 0;     // colours, block width (band width), block steps
  const double* Ablk = nullptr;        // [c][m][b][b]
  const double* Bblk = nullptr;        // [c][m][b][b]
  const int32_t* nblk = nullptr;       // [c] blocks in use (0 for an empty colour)
  const int32_t* cnt = nullptr;        // [c] molecules of the colour
  const double* B0 = nullptr;          // [c][b][b] general start factor (nullptr: B_0 = sqrt|c| I)
  int32_t rcap = 0;                    // reflector slots per colour
  double* AB = nullptr;                // [c][nmax][2b+1]
  double* RV = nullptr;                // [c][rcap][b]
  double* RT = nullptr;                // [c][rcap]
  int32_t* RR0 = nullptr;              // [c][rcap]
  int32_t* sweep_off = nullptr;        // [c][nmax+1]
  double *d = nullptr, *e = nullptr;   // [c][nmax] tridiagonal
  float* lam32 = nullptr;              // [c][nmax] FP32 shifts
  double* tnorm = nullptr;             // [c]
  double* U = nullptr;                 // [c][nmax][nmax] eigenvectors of the tridiagonal
  double* F = nullptr;                 // [c][5][nmax][nmax] LU scratch
  double* lam = nullptr;               // [c][nmax] eigenvalues
  double* X0 = nullptr;                // [c][nmax][b] Q_band^T E_1 B_0
  double* Y = nullptr;                 // [c][nmax][b] U^T X0
  double* wgt = nullptr;               // [c][nmax] ||Y_k||^2
  int32_t* status = nullptr;           // [c]
  int32_t* flag = nullptr;             // [c][nmax] eigenvalues left to the sequential phase
  const int32_t* gid = nullptr;        // [c] the colour's id for its inverse-iteration start vectors
                                       // (nullptr: its index here; a colour subset passes the full
                                       // call's numbering so that its results do not change)
};

css_status css_eigen_ritz(css_ctx* ctx, const EigArgs& a, cudaStream_t st);
css_status css_eigen_z(css_ctx* ctx, const EigArgs& a, const int32_t* sys_of_colour, const double* mu,
                       const double* kT, double* Z, cudaStream_t st, int fn = 0);
// after css_eigen_ritz: YV = U^T Q_band^T V for another n x b block per colour ([c][nmax][b], V is
// overwritten by Q_band^T V), in the same order of operations that gives Y from E_1 B_0; scratch
// receives the row norms
css_status css_eigen_project(css_ctx* ctx, const EigArgs& a, double* V, double* YV, double* scratch, cudaStream_t st);
