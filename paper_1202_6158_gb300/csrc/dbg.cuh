// dbg.cuh -- device-side index checks of the DI_DEBUG build (libditer_debug.so).
//
// In a DI_DEBUG build, DI_CHECK(cond, code, idx) evaluates cond; when it is false it records
// the first failure of the translation unit in a device word, (code << 48) | (idx & 2^48-1),
// and returns false so that the caller skips the access (never a trap).  The host reads and
// clears the word after each solve (dbg_take_*), and the call returns DI_EKERNEL naming the
// check.  In the release build DI_CHECK is the constant true and cond is not evaluated.
//
// Codes: 1 a scan list append beyond its warp's region; 2 a push list position beyond its
// sub-chunk's region; 3 a listed node id outside [0, n); 4 a pushed-to column outside
// [0, n); 5 a pull link endpoint outside [0, n); 99 the self-test.
#pragma once

#include <cuda_runtime.h>

namespace diter {
namespace {

#ifdef DI_DEBUG
__device__ unsigned long long g_dbg_word;
__device__ __forceinline__ bool dbg_ok(bool ok, unsigned code, long long idx) {
    if (!ok)
        atomicCAS(&g_dbg_word, 0ull,
                  ((unsigned long long)code << 48) | ((unsigned long long)idx & 0xffffffffffffull));
    return ok;
}
#define DI_CHECK(cond, code, idx) ::diter::dbg_ok((cond), (code), (long long)(idx))
// the translation unit's word, cleared
inline unsigned long long dbg_take_word() {
    unsigned long long w = 0, z = 0;
    if (cudaMemcpyFromSymbol(&w, g_dbg_word, sizeof(w)) != cudaSuccess) return 0;
    if (w) cudaMemcpyToSymbol(g_dbg_word, &z, sizeof(z));
    return w;
}
#else
#define DI_CHECK(cond, code, idx) true
#endif

}  // namespace
}  // namespace diter
