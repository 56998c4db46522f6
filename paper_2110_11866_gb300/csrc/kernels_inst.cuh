// Explicit instantiations of the scan kernel, one translation unit per variant so that the build
// compiles them in parallel. Each unit defines `const void* <name>(int K)` returning the kernel for
// one of the built term counts (2, 3, 4, 6, 8, 12) or nullptr.
#pragma once

#include "plan_internal.h"
#include "scan_kernel.cuh"
#include "wscan_kernel.cuh"

#define MSFT_INST(NAME, R, CV, FORM, OUT, ASFT, ITEMS)                                   \
  namespace msft {                                                                      \
  const void* NAME(int K) {                                                             \
    switch (K) {                                                                        \
      case 2: return (const void*)&scan_kernel<Cfg<R, CV, 2, FORM, OUT, ASFT, ITEMS>>;   \
      case 3: return (const void*)&scan_kernel<Cfg<R, CV, 3, FORM, OUT, ASFT, ITEMS>>;   \
      case 4: return (const void*)&scan_kernel<Cfg<R, CV, 4, FORM, OUT, ASFT, ITEMS>>;   \
      case 6: return (const void*)&scan_kernel<Cfg<R, CV, 6, FORM, OUT, ASFT, ITEMS>>;   \
      case 8: return (const void*)&scan_kernel<Cfg<R, CV, 8, FORM, OUT, ASFT, ITEMS>>;   \
      case 12: return (const void*)&scan_kernel<Cfg<R, CV, 12, FORM, OUT, ASFT, ITEMS>>; \
      default: return nullptr;                                                          \
    }                                                                                   \
  }                                                                                     \
  }

// Warp-independent kernel of a rotating-form variant (window rows): `const void* NAME(int K)`.
#define MSFT_INST_W(NAME, R, CV, OUT, ASFT, ITEMS)                                                  \
  namespace msft {                                                                                 \
  const void* NAME(int K) {                                                                        \
    switch (K) {                                                                                   \
      case 2: return (const void*)&wscan_kernel<Cfg<R, CV, 2, FORM_RF, OUT, ASFT, ITEMS>>;         \
      case 3: return (const void*)&wscan_kernel<Cfg<R, CV, 3, FORM_RF, OUT, ASFT, ITEMS>>;         \
      case 4: return (const void*)&wscan_kernel<Cfg<R, CV, 4, FORM_RF, OUT, ASFT, ITEMS>>;         \
      case 6: return (const void*)&wscan_kernel<Cfg<R, CV, 6, FORM_RF, OUT, ASFT, ITEMS>>;         \
      case 8: return (const void*)&wscan_kernel<Cfg<R, CV, 8, FORM_RF, OUT, ASFT, ITEMS>>;         \
      case 12: return (const void*)&wscan_kernel<Cfg<R, CV, 12, FORM_RF, OUT, ASFT, ITEMS>>;       \
      default: return nullptr;                                                                     \
    }                                                                                              \
  }                                                                                                \
  }
