// Checks f64_to_f32_rn (the library's integer-pipe FP64 -> FP32 rounding) against
// the conversion instruction __double2float_rn, bit for bit, on 2^24 values per
// launch: random bit patterns over the normal FP32 range, exact ties (dropped bits
// exactly half an FP32 unit, kept fraction even and odd), values just above and
// below ties, carries into the exponent, zeros, and out-of-range values.
// Prints the number of mismatches and exits 1 when there is any.
#include <cstdio>
#include <cstdint>

#include "f64conv.cuh"

__device__ uint64_t splitmix(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__global__ void check(uint64_t seed, unsigned long long* bad, unsigned long long* first) {
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t r = splitmix(seed * 0x100000000ull + i);
    uint64_t bits;
    const int kind = int(i & 7);
    // exponent within (and a little beyond) the normal FP32 range
    const uint64_t e = 1023 - 130 + (splitmix(r) % 262);
    const uint64_t sign = (r >> 63) << 63;
    uint64_t frac = r & 0xfffffffffffffull;
    if (kind == 1) frac = (frac & ~0x1fffffffull) | 0x10000000ull;                 // tie
    if (kind == 2) frac = (frac & ~0x1fffffffull) | 0x10000001ull;                 // just above a tie
    if (kind == 3) frac = (frac & ~0x1fffffffull) | 0x0fffffffull;                 // just below a tie
    if (kind == 4) frac = 0xfffffffffffffull - (r & 0xfffffffull);                 // near a carry
    bits = sign | (e << 52) | frac;
    if (kind == 5 && (r & 0xff) == 0) bits = sign;                                 // zero
    const double x = __longlong_as_double(static_cast<long long>(bits));
    const float a = f64_to_f32_rn(x), b = __double2float_rn(x);
    if (__float_as_uint(a) != __float_as_uint(b)) {
        if (atomicAdd(bad, 1ull) == 0ull) *first = bits;
    }
}

int main() {
    unsigned long long *bad, *first;
    cudaMallocManaged(&bad, sizeof(unsigned long long));
    cudaMallocManaged(&first, sizeof(unsigned long long));
    *bad = 0, *first = 0;
    for (uint64_t s = 1; s <= 8; ++s) check<<<65536, 256>>>(s, bad, first);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        printf("launch failed\n");
        return 2;
    }
    printf("mismatches %llu first %016llx\n", *bad, *first);
    return *bad ? 1 : 0;
}
