// Host-side check of the structured trend's shared-memory layout and geometry
// blocks (sww_tile.cuh) for every working precision and patch side: the bulk
// copies need 16-byte aligned, 16-byte multiple blocks and buffers, the mbarriers
// 8-byte alignment, the element copies word-aligned destinations, and the
// dynamic plus static shared memory must fit a block (and five blocks of 8 x 8
// FP32 tiles an SM, as the kernel is built for).  Prints "tile layout ok".
#include <cstdint>
#include <cstdio>

#include "sww_core.cuh"
#include "sww_kernels.h"
#include "sww_stage.h"
#include "tile.h"

namespace sww {
namespace {
#include "bulk.cuh"
#include "sww_bodies.cuh"
#include "sww_tile.cuh"

int failures = 0;

void expect(bool ok, const char* what, const char* name, int p) {
    if (!ok) {
        std::printf("FAIL %s (%s, p = %d)\n", what, name, p);
        ++failures;
    }
}

template <class R, int P>
void check(const char* name) {
    using T = Tile<R, P>;
    using G = TileGeo<R, P>;
    const size_t rs = sizeof(R);
    expect(G::BYTES % 16 == 0 && size_t(G::WORDS) * rs == G::BYTES, "geometry block a 16-byte multiple", name, P);
    expect(G::AI + G::PP <= G::WORDS, "geometry block holds every field", name, P);
    expect(T::OFF_GEO % 16 == 0 && T::OFF_STG % 16 == 0 && T::STAGED % 16 == 0, "bulk-copy buffers 16-byte aligned",
           name, P);
    expect(T::ST_U % rs == 0 && T::ST_NFW % 4 == 0 && T::ST_EFW % 4 == 0, "element-copy destinations aligned", name, P);
    expect(T::ST_EF + 3 * T::NN <= T::STAGED, "staged fields inside their buffer", name, P);
    expect(T::OFF_F % rs == 0 && T::OFF_Q % rs == 0 && T::OFF_Q + rs * 2 * T::NN <= T::OFF_BAR, "F and q placed",
           name, P);
    expect(T::OFF_BAR % 8 == 0 && T::OFF_BAR + 16 <= T::BYTES, "mbarriers aligned and inside", name, P);
    const size_t stat = 12 * sizeof(DevLevelT<R>);   // the level records of a block
    expect(T::BYTES + stat <= 227 * 1024, "shared memory of one block", name, P);
    std::printf("%s p=%2d: geometry block %6u B, dynamic %6zu B, static %5zu B\n", name, P, G::BYTES,
                size_t(T::BYTES), stat);
}
}  // namespace
}  // namespace sww

int main() {
    using namespace sww;
    check<float, 4>("fp32");
    check<float, 8>("fp32");
    check<float, 16>("fp32");
    check<double, 4>("fp64");
    check<double, 8>("fp64");
    check<double, 16>("fp64");
    // five resident blocks of 8 x 8 FP32 tiles per SM (228 KB, 1 KB reserved per block)
    const size_t per_block = Tile<float, 8>::BYTES + 12 * sizeof(DevLevelT<float>) + 1024;
    expect(5 * per_block <= 228 * 1024, "five 8 x 8 FP32 blocks per SM", "fp32", 8);
    if (failures == 0) std::printf("tile layout ok\n");
    return failures == 0 ? 0 : 1;
}
