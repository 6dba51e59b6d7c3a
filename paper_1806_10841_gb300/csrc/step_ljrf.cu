// Force/step kernels of the water-like model (three sites per molecule, Lennard-Jones +
// reaction-field Coulomb between molecules, harmonic bonds and angle), in their own
// translation unit so the two models compile in parallel.
#include "step_impl.cuh"

namespace adress {

cudaError_t launch_step_ljrf(const Sys& s, const Bufs& b, int precision, int mode, int energy, cudaStream_t st) {
  if (s.NA != 3) return cudaErrorInvalidValue;
  if (precision == ADRESS_FP64) launch_step_na<P64, 3, 1, false>(s, b, mode, energy, st);
  else launch_step_na<P32, 3, 1, false>(s, b, mode, energy, st);
  return cudaGetLastError();
}

}  // namespace adress
