// Step kernels of energy interpolation (H-AdResS, Eq. Hmix) for both models: pair weight
// (l_a + l_b)/2 and the drift force on hybrid molecules.  A translation unit of their own so
// that they compile in parallel with the force-interpolation kernels.
#include "step_impl.cuh"

namespace adress {

template <class P>
static void launch_hadress_p(const Sys& s, const Bufs& b, int mode, int energy, cudaStream_t st) {
  if (s.nb_model == 1) {
    launch_step_na<P, 3, 1, true>(s, b, mode, energy, st);
    return;
  }
  switch (s.NA) {
    case 1: launch_step_na<P, 1, 0, true>(s, b, mode, energy, st); break;
    case 2: launch_step_na<P, 2, 0, true>(s, b, mode, energy, st); break;
    case 3: launch_step_na<P, 3, 0, true>(s, b, mode, energy, st); break;
    default: launch_step_na<P, 4, 0, true>(s, b, mode, energy, st); break;
  }
}

cudaError_t launch_step_hadress(const Sys& s, const Bufs& b, int precision, int mode, int energy, cudaStream_t st) {
  if (s.nb_model == 1 && s.NA != 3) return cudaErrorInvalidValue;
  if (precision == ADRESS_FP64) launch_hadress_p<P64>(s, b, mode, energy, st);
  else launch_hadress_p<P32>(s, b, mode, energy, st);
  return cudaGetLastError();
}

}  // namespace adress
