// Division by a run-time divisor through a precomputed reciprocal (host and
// device; no CUDA headers, so the CPU tests compile it with a plain C++
// compiler).
//
// For d >= 1 let r = floor((2^32 - 1) / d).  For n < 2^31 the estimate
// q' = floor(n r / 2^32) is the quotient q = floor(n / d) or q - 1: from
// (2^32 - 1 - d) / d < r < 2^32 / d it follows that
// n / d - n (1 + d) / (d 2^32) < n r / 2^32 <= n / d, and n (1 + d) / (d 2^32)
// < 1 whenever n < 2^31 (d / (1 + d) >= 1/2).  One compare of the remainder
// against d corrects it: a multiply-high and two integer instructions
// instead of a ~20-instruction 32-bit division.
#pragma once

#ifdef __CUDACC__
#define PP_FASTDIV_HD __host__ __device__ __forceinline__
#else
#define PP_FASTDIV_HD inline
#endif

namespace pp {

PP_FASTDIV_HD unsigned fdiv_rcp(unsigned d) { return d ? 0xFFFFFFFFu / d : 0u; }

PP_FASTDIV_HD unsigned fdiv(unsigned n, unsigned d, unsigned r) {
#ifdef __CUDA_ARCH__
    unsigned q = __umulhi(n, r);
#else
    unsigned q = (unsigned)(((unsigned long long)n * r) >> 32);
#endif
    if (n - q * d >= d) ++q;
    return q;
}

}  // namespace pp
