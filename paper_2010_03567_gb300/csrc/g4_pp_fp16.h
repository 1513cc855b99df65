/* g4_pp_fp16.h -- constants of the FP16x2 candidate test of the particle-particle phase
 * (g4_pp.cuh).  For a group whose sinks lie within R r_cut of the group centre (per axis),
 * FP16 positions relative to the centre in units of r_cut err by at most
 *   e = (G4_PP_FP16_EA R + G4_PP_FP16_EB) / G4_PP_FP16_ULP          per axis,
 * so a pair inside r_cut has a computed r^2 / r_cut^2 of at most 1 + 2 sqrt(3) e + 3 e^2 plus
 * the rounding of the FP16 sums; the test keeps every source with
 *   r^2 / r_cut^2 < (1 + G4_PP_FP16_C1 e + G4_PP_FP16_C2 e^2) G4_PP_FP16_SLACK_MUL
 *                   + G4_PP_FP16_SLACK_ADD                            (rounded up in FP16),
 * and groups wider than G4_PP_FP16_RMAX r_cut skip the test (every staged source is a
 * candidate).
 * Before that test, staged sources farther than r_cut from the sinks' bounding box are dropped
 * (FP32 offsets from the group centre, half extents = the sinks' largest |offset| per axis):
 * kept when the squared distance is <= r_cut^2 G4_PP_PRUNE_MARGIN, for groups within
 * G4_PP_PRUNE_RMAX r_cut of their centre (wider groups keep every staged source).
 * Plain macros: the CPU tests of both bounds read them from this file. */
#ifndef G4_PP_FP16_H
#define G4_PP_FP16_H
#define G4_PP_FP16_RMAX 2048.0f
#define G4_PP_FP16_EA 2.0f
#define G4_PP_FP16_EB 2.0f
#define G4_PP_FP16_ULP 2048.0f
#define G4_PP_FP16_C1 3.4642f
#define G4_PP_FP16_C2 3.0f
#define G4_PP_FP16_SLACK_MUL 1.002f
#define G4_PP_FP16_SLACK_ADD 0.002f
#define G4_PP_PRUNE_RMAX 64.0f
#define G4_PP_PRUNE_MARGIN 1.0002f
#endif
