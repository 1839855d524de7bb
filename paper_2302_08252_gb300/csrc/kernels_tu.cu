// Instantiates the transport kernels for one (mode, layout) pair; compiled once
// per pair with -DET_MODE=<0 strict|1 fast> -DET_LAYOUT=<0..3>.  Strict
// objects are built with --fmad=false so that every FP32 operation of the toy
// model is a separately rounded IEEE operation.
#include "kernels.cuh"
#include "registry.h"

#ifndef ET_MODE
#error "ET_MODE must be defined"
#endif
#ifndef ET_LAYOUT
#error "ET_LAYOUT must be defined"
#endif

#define ET_CAT2(a, b, c) et_register_kernels_##a##_##b
#define ET_CAT(a, b) ET_CAT2(a, b, x)

namespace et {

template <bool INSTR>
static void fill(KernelSet* ks) {
  constexpr int M = ET_MODE, L = ET_LAYOUT;
  ks->step[INSTR][1][EM] = (const void*)k_step<EM, M, L, INSTR, true>;
  ks->step[INSTR][1][EP] = (const void*)k_step<EP, M, L, INSTR, true>;
  ks->step[INSTR][1][GAM] = (const void*)k_step<GAM, M, L, INSTR, true>;
  ks->step[INSTR][0][EM] = (const void*)k_step<EM, M, L, INSTR, false>;
  ks->step[INSTR][0][EP] = (const void*)k_step<EP, M, L, INSTR, false>;
  ks->step[INSTR][0][GAM] = (const void*)k_step<GAM, M, L, INSTR, false>;
  ks->persistent[INSTR][1] = (const void*)k_persistent<M, L, INSTR, true>;
  ks->persistent[INSTR][0] = (const void*)k_persistent<M, L, INSTR, false>;
}

template <bool DENSE>
static void fill_split(KernelSet* ks) {
  constexpr int M = ET_MODE, L = ET_LAYOUT, D = DENSE ? 1 : 0;
  ks->transport[D][EM] = (const void*)k_transport<EM, M, L, DENSE>;
  ks->transport[D][EP] = (const void*)k_transport<EP, M, L, DENSE>;
  ks->transport[D][GAM] = (const void*)k_transport<GAM, M, L, DENSE>;
  ks->interact[D][EM] = (const void*)k_interact<EM, M, L, DENSE>;
  ks->interact[D][EP] = (const void*)k_interact<EP, M, L, DENSE>;
  ks->interact[D][GAM] = (const void*)k_interact<GAM, M, L, DENSE>;
}

}  // namespace et

extern "C" void ET_CAT(ET_MODE, ET_LAYOUT)(et::KernelSet* ks) {
  et::fill<false>(ks);
#if ET_MODE == 0
  et::fill<true>(ks);  // the instrumented build counts accesses of the strict model
#endif
  ks->inject[1] = (const void*)et::k_inject<ET_LAYOUT, true>;
  ks->inject[0] = (const void*)et::k_inject<ET_LAYOUT, false>;
  ks->mark_present[1] = (const void*)et::k_mark_present<ET_LAYOUT, true>;
  ks->mark_present[0] = (const void*)et::k_mark_present<ET_LAYOUT, false>;
  et::fill_split<true>(ks);
  et::fill_split<false>(ks);
}
