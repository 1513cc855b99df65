// g4_fmm_variant.cu -- one (order, TreePM) variant of the FMM dual walk (g4_fmm.cuh).
// The build compiles this file once per variant with -DG4_FMM_P=<order> -DG4_FMM_TREEPM=<0|1>,
// so that the heavily unrolled kernels of the eight variants compile in parallel; compiled
// without those macros it holds all of them.
#include "g4_fmm.cuh"

#if defined(G4_FMM_P) && defined(G4_FMM_TREEPM)
template void g4fmm::run_variant<G4_FMM_P, (G4_FMM_TREEPM != 0)>(const g4fmm::FmmArgs &, bool, cudaStream_t);
#else
template void g4fmm::run_variant<2, false>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<2, true>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<3, false>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<3, true>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<4, false>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<4, true>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<5, false>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<5, true>(const g4fmm::FmmArgs &, bool, cudaStream_t);
#endif
