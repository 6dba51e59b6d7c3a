// Launchers of the MD-step kernels (step_impl.cuh): the prologue for every molecule size
// and the force-interpolation step kernels of the WCA model; the water-like model's kernels
// are instantiated in step_ljrf.cu and the energy-interpolation ones in step_hadress.cu.
#include "step_impl.cuh"

namespace adress {

cudaError_t launch_step_ljrf(const Sys& s, const Bufs& b, int precision, int mode, int energy, cudaStream_t st);
cudaError_t launch_step_hadress(const Sys& s, const Bufs& b, int precision, int mode, int energy, cudaStream_t st);

template <class P, int NA>
static void launch_prologue_na(const Sys& s, const Bufs& b, int integrate, cudaStream_t st) {
  const int blocks = ceil_div((long long)s.M * kGroup, s.force_block);
  if (s.nbox > 1) {
    if (integrate) k_prologue<P, NA, true, true><<<blocks, s.force_block, 0, st>>>(s, b);
    else k_prologue<P, NA, false, true><<<blocks, s.force_block, 0, st>>>(s, b);
  } else {
    if (integrate) k_prologue<P, NA, true, false><<<blocks, s.force_block, 0, st>>>(s, b);
    else k_prologue<P, NA, false, false><<<blocks, s.force_block, 0, st>>>(s, b);
  }
}

template <class P>
static void launch_prologue_p(const Sys& s, const Bufs& b, int integrate, cudaStream_t st) {
  switch (s.NA) {
    case 1: launch_prologue_na<P, 1>(s, b, integrate, st); break;
    case 2: launch_prologue_na<P, 2>(s, b, integrate, st); break;
    case 3: launch_prologue_na<P, 3>(s, b, integrate, st); break;
    default: launch_prologue_na<P, 4>(s, b, integrate, st); break;
  }
}

cudaError_t launch_com(const Sys& s, const Bufs& b, int precision, int integrate, cudaStream_t st, DecideArgs da) {
  if (precision == ADRESS_FP64) launch_prologue_p<P64>(s, b, integrate, st);
  else launch_prologue_p<P32>(s, b, integrate, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? launch_decide(s, b, da, st) : e;
}

template <class P>
static void launch_step_p(const Sys& s, const Bufs& b, int mode, int energy, cudaStream_t st) {
  switch (s.NA) {
    case 1: launch_step_na<P, 1, 0, false>(s, b, mode, energy, st); break;
    case 2: launch_step_na<P, 2, 0, false>(s, b, mode, energy, st); break;
    case 3: launch_step_na<P, 3, 0, false>(s, b, mode, energy, st); break;
    default: launch_step_na<P, 4, 0, false>(s, b, mode, energy, st); break;
  }
}

cudaError_t launch_step(const Sys& s, const Bufs& b, int precision, int mode, int energy, cudaStream_t st,
                        DecideArgs da) {
  cudaError_t e;
  if (s.scheme == 1) {
    e = launch_step_hadress(s, b, precision, mode, energy, st);
  } else if (s.nb_model == 1) {
    e = launch_step_ljrf(s, b, precision, mode, energy, st);
  } else {
    if (precision == ADRESS_FP64) launch_step_p<P64>(s, b, mode, energy, st);
    else launch_step_p<P32>(s, b, mode, energy, st);
    e = cudaGetLastError();
  }
  return (e == cudaSuccess && mode == MODE_FUSED) ? launch_decide(s, b, da, st) : e;
}

}  // namespace adress
