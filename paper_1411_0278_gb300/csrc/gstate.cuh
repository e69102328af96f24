// Per-system GMRES state of the device-side solver and the size of the state buffer
// (shared by the solver and the static-storage entry point, which sizes its slot from it).
#pragma once

#include <stddef.h>

namespace gbi {

struct GDev {
  int j;          // Arnoldi index of the vector being expanded
  int active;     // 1 while the current cycle continues
  int iters;      // inner iterations of the current inner solve
  int kdim;       // Krylov dimension reached in the current cycle
  int converged;  // relative residual estimate <= tol
  int breakdown;  // happy breakdown (exact solution in the Krylov space)
  int max_iter, m;
  int enabled;    // refinement: this system still needs a correction
  int it0;        // iterations already counted (device-decided solve)
  double bnorm, tol, res, beta, inv_hn;
  double nb;      // |b_s| (reference of the refinement residual)
  double rel;     // |b_s - A q_s| / |b_s|
  double inv_bnorm, inv_nb;   // 1 / bnorm, 1 / nb (0 for a zero norm)
};

// Arnoldi dot-product chunks per system: one block per (system, component row) for fewer
// than 64 systems, else one per system.
constexpr int arnoldi_chunks(int S, int h) { return S >= 64 ? 1 : h; }

// Doubles of the state buffer for restart length m, S systems and CH chunks per system:
// the per-system states, Hessenberg columns and Givens data, the chunk partial sums, the
// fused step's block partials and the barrier / counter words.
constexpr size_t gstate_doubles(int m, int S, int CH, int fused_blocks) {
  return (size_t)S * (sizeof(GDev) / sizeof(double) + 1) + (size_t)S * ((size_t)(m + 1) * m + 6 * (size_t)(m + 1) + 1) +
         (size_t)S * CH * (2 * (size_t)(m + 1) + 1) + (size_t)fused_blocks * (2 * (size_t)(m + 1) + 1) + 24 +
         ((size_t)S + 1) / 2 + 1;
}

}  // namespace gbi
