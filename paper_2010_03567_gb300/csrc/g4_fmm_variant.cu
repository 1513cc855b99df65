// g4_fmm_variant.cu -- one (order, TreePM, interaction type) variant of the FMM dual walk
// (g4_fmm.cuh).  The build compiles this file once per variant with -DG4_FMM_P=<order>
// -DG4_FMM_TREEPM=<0|1> (and -DG4_FMM_FP64=1 for the FP64 reference mode, order 4), so that
// the heavily unrolled kernels of the variants compile in parallel; compiled without those
// macros it holds all of them.
#include "g4_fmm.cuh"

#if defined(G4_FMM_P) && defined(G4_FMM_TREEPM)
#if defined(G4_FMM_FP64) && G4_FMM_FP64
template void g4fmm::run_variant<G4_FMM_P, (G4_FMM_TREEPM != 0), double>(const g4fmm::FmmArgs &, bool, cudaStream_t);
#else
template void g4fmm::run_variant<G4_FMM_P, (G4_FMM_TREEPM != 0), float>(const g4fmm::FmmArgs &, bool, cudaStream_t);
#endif
#else
template void g4fmm::run_variant<2, false, float>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<2, true, float>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<3, false, float>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<3, true, float>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<4, false, float>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<4, true, float>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<5, false, float>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<5, true, float>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<4, false, double>(const g4fmm::FmmArgs &, bool, cudaStream_t);
template void g4fmm::run_variant<4, true, double>(const g4fmm::FmmArgs &, bool, cudaStream_t);
#endif
