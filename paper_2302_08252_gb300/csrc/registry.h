// Kernel registry: each (mode, layout) translation unit fills one KernelSet
// with its kernels' entry addresses; the host side launches through these.
#pragma once

namespace et {

struct KernelSet {
  const void* step[2][2][3];     // [instrumented][dense][type]
  const void* persistent[2][2];  // [instrumented][dense]
  const void* inject[2];         // [dense]
  const void* mark_present[2];   // [dense] serving: events with tracks in the buffers
  const void* transport[2][3];   // split form, not instrumented: [dense][type]
  const void* interact[2][3];    // split form, not instrumented: [dense][type]
};

}  // namespace et

extern "C" {
void et_register_kernels_0_0(et::KernelSet*);
void et_register_kernels_0_1(et::KernelSet*);
void et_register_kernels_0_2(et::KernelSet*);
void et_register_kernels_0_3(et::KernelSet*);
void et_register_kernels_0_4(et::KernelSet*);
void et_register_kernels_0_5(et::KernelSet*);
void et_register_kernels_0_6(et::KernelSet*);
void et_register_kernels_0_7(et::KernelSet*);
void et_register_kernels_1_0(et::KernelSet*);
void et_register_kernels_1_1(et::KernelSet*);
void et_register_kernels_1_2(et::KernelSet*);
void et_register_kernels_1_3(et::KernelSet*);
void et_register_kernels_1_4(et::KernelSet*);
void et_register_kernels_1_5(et::KernelSet*);
void et_register_kernels_1_6(et::KernelSet*);
void et_register_kernels_1_7(et::KernelSet*);
}
