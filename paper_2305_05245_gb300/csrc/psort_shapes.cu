// psort_shapes.cu -- the table of launch shapes compiled besides the automatic
// one (psort_shape.cu, one object per shape).
#include "psort_internal.h"

namespace ps {

extern const ShapeEntry shape_u32_e16_t128, shape_u32_e16_t256, shape_u32_e16_t512, shape_u32_e32_t128,
    shape_u32_e32_t256, shape_u32_e32_t512, shape_u64_e16_t128, shape_u64_e16_t256, shape_u64_e16_t512,
    shape_u64_e32_t128, shape_u64_e32_t512;

static const ShapeEntry* const kShapes[] = {
    &shape_u32_e16_t128, &shape_u32_e16_t256, &shape_u32_e16_t512, &shape_u32_e32_t128, &shape_u32_e32_t256,
    &shape_u32_e32_t512, &shape_u64_e16_t128, &shape_u64_e16_t256, &shape_u64_e16_t512, &shape_u64_e32_t128,
    &shape_u64_e32_t512, nullptr};

const ShapeEntry* find_shape(int bits, int items, int threads)
{
    for (const ShapeEntry* const* e = kShapes; *e; e++)
        if ((*e)->bits == bits && (*e)->items == items && (*e)->threads == threads) return *e;
    return nullptr;
}

const ShapeEntry* const* all_shapes() { return kShapes; }

}  // namespace ps
