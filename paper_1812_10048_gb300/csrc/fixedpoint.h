// Exact conversion of an FP32 value to a signed count of 2^-32 units, rounded
// to nearest (ties to even), in integer arithmetic only.  The result equals
// rounding the exact product x * 2^32 to the nearest integer: x = m 2^(e-150)
// with a 24-bit m, so x 2^32 = m 2^(e-118), a left shift when e >= 118 and a
// right shift with round-half-even below.  |x| >= 2^31 saturates to the int64
// range, a NaN gives 0.  Plain C++: the same code builds for the host (tests)
// and the device.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define DPMM_HD __host__ __device__ __forceinline__
#else
#define DPMM_HD static inline
#endif

DPMM_HD int64_t fixed32_from_float(float x) {
    uint32_t b;
    memcpy(&b, &x, sizeof(b));
    const uint32_t e = (b >> 23) & 0xFFu;
    const bool neg = (b >> 31) != 0u;
    if (e == 0xFFu) {
        if (b & 0x7FFFFFu) return 0;                                       // NaN
        return neg ? (int64_t)(-9223372036854775807LL - 1) : (int64_t)9223372036854775807LL;
    }
    if (e < 94u) return 0;               // |x| < 2^-33: x 2^32 < 1/2 (zero and subnormals too)
    const uint64_t m = (uint64_t)((b & 0x7FFFFFu) | 0x800000u);
    uint64_t q;
    if (e >= 118u) {
        if (e > 157u)                    // |x| >= 2^31: beyond int64 after scaling
            return neg ? (int64_t)(-9223372036854775807LL - 1) : (int64_t)9223372036854775807LL;
        q = m << (e - 118u);
    } else {
        const uint32_t k = 118u - e;     // 1 .. 24
        const uint64_t half = 1ull << (k - 1u);
        const uint64_t r = m & ((1ull << k) - 1ull);
        q = m >> k;
        if (r > half || (r == half && (q & 1ull))) ++q;
    }
    return neg ? -(int64_t)q : (int64_t)q;
}
