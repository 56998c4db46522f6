// Explicit instantiations of the scan kernel, one translation unit per variant so that the build
// compiles them in parallel. Each unit defines `const void* <name>(int K)` returning the kernel for
// one of the built term counts (2, 3, 4, 6, 8, 12) or nullptr.
#pragma once

#include "plan_internal.h"
#include "scan_kernel.cuh"

#define MSFT_INST(NAME, R, CR, FORM, OUT, ASFT, ITEMS)                                   \
  namespace msft {                                                                      \
  const void* NAME(int K) {                                                             \
    switch (K) {                                                                        \
      case 2: return (const void*)&scan_kernel<Cfg<R, CR, 2, FORM, OUT, ASFT, ITEMS>>;   \
      case 3: return (const void*)&scan_kernel<Cfg<R, CR, 3, FORM, OUT, ASFT, ITEMS>>;   \
      case 4: return (const void*)&scan_kernel<Cfg<R, CR, 4, FORM, OUT, ASFT, ITEMS>>;   \
      case 6: return (const void*)&scan_kernel<Cfg<R, CR, 6, FORM, OUT, ASFT, ITEMS>>;   \
      case 8: return (const void*)&scan_kernel<Cfg<R, CR, 8, FORM, OUT, ASFT, ITEMS>>;   \
      case 12: return (const void*)&scan_kernel<Cfg<R, CR, 12, FORM, OUT, ASFT, ITEMS>>; \
      default: return nullptr;                                                          \
    }                                                                                   \
  }                                                                                     \
  }
