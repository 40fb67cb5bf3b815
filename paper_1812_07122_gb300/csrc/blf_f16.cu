// K1 kernel instantiations of the F16 form, radii 0..16 (single-image, joint and
// batched drivers).  Split by precision so the three translation units compile in parallel.
#include "blf_tile.cuh"

namespace blfls {
namespace {

template <int R>
TiledFn pick_tiled_f16(int r, bool range)
{
    if constexpr (R > kMaxTemplR) {
        return nullptr;
    } else {
        if (r != R) return pick_tiled_f16<R + 1>(r, range);
        return range ? k1_blf<R, true, 1> : k1_blf<R, false, 1>;
    }
}

template <int R>
BatchFn pick_batch_f16(int r, bool range)
{
    if constexpr (R > kMaxTemplR) {
        return nullptr;
    } else {
        if (r != R) return pick_batch_f16<R + 1>(r, range);
        return range ? k1_blf_batch<R, true, 1> : k1_blf_batch<R, false, 1>;
    }
}

template <int R>
JointFn pick_joint_f16(int r)
{
    if constexpr (R > kMaxTemplR) {
        return nullptr;
    } else {
        if (r != R) return pick_joint_f16<R + 1>(r);
        return k1_blf_joint<R, 1>;
    }
}

}  // namespace

BLFLS_DCHECK_TU(blf_f16)

JointFn pick_joint_f16_entry(int r) { return pick_joint_f16<0>(r); }
TiledFn pick_tiled_f16_entry(int r, bool range) { return pick_tiled_f16<0>(r, range); }
BatchFn pick_batch_f16_entry(int r, bool range) { return pick_batch_f16<0>(r, range); }

}  // namespace blfls
