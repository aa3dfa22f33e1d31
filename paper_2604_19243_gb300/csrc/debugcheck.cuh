// Bounds checks of the FMM_DEBUG build (libfmm_debug.so, compiled with -DFMM_DEBUG).  A failed
// check ORs its bit into the debug word of its translation unit, and the caller skips the access
// it guards: nothing traps.  fmm_debug_check reads and clears the words of every unit.  In the
// normal build dbg_ok is `true` and the checks compile away.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fmm.h"

namespace fmm {

// bits of the debug word: the fmm_debug_bits of include/fmm.h (also those of the table
// validator, validate_tree in tree.cu)
enum : uint32_t {
    kDbgPerm = FMM_DEBUG_PERM,
    kDbgLeaf = FMM_DEBUG_LEAF,
    kDbgUList = FMM_DEBUG_ULIST,
    kDbgKeys = FMM_DEBUG_KEYS,
    kDbgTree = FMM_DEBUG_TREE,
    kDbgClass = FMM_DEBUG_CLASS,
    kDbgOrder = FMM_DEBUG_ORDER,
    kDbgP2P = FMM_DEBUG_P2P,
    kDbgScatter = FMM_DEBUG_SCATTER,
    kDbgSort = FMM_DEBUG_SORT,
};

#ifdef FMM_DEBUG
static __device__ unsigned int g_fmm_debug_word;
__device__ __forceinline__ bool dbg_ok(bool cond, uint32_t bit) {
    if (!cond) atomicOr(&g_fmm_debug_word, bit);
    return cond;
}
#define FMM_DEBUG_UNIT(name)                                                           \
    uint32_t debug_word_##name(bool clear) {                                           \
        unsigned int v = 0, z = 0;                                                     \
        if (cudaMemcpyFromSymbol(&v, g_fmm_debug_word, sizeof(v)) != cudaSuccess) {    \
            cudaGetLastError();                                                        \
            return 0;                                                                  \
        }                                                                              \
        if (clear) cudaMemcpyToSymbol(g_fmm_debug_word, &z, sizeof(z));                \
        return v;                                                                      \
    }
#else
__device__ __forceinline__ bool dbg_ok(bool, uint32_t) { return true; }
#define FMM_DEBUG_UNIT(name) \
    uint32_t debug_word_##name(bool) { return 0; }
#endif

}  // namespace fmm
