// psort_shape.cu -- the keys-only pipeline for one launch shape other than the
// automatic one.  Compiled once per shape with
//   -DPS_SHAPE_BITS=32|64 -DPS_SHAPE_ITEMS=16|32 -DPS_SHAPE_THREADS=128|256|512
// (see build.py); each object defines one ShapeEntry that psort_shapes.cu
// lists.  Tile sort and chunk merge share the shape: block_threads CTAs with
// items_per_thread keys each, so tile and chunk capacity are equal.
#include <type_traits>

#include "psort_pipeline.cuh"

#if !defined(PS_SHAPE_BITS) || !defined(PS_SHAPE_ITEMS) || !defined(PS_SHAPE_THREADS)
#error "psort_shape.cu is compiled with PS_SHAPE_BITS, PS_SHAPE_ITEMS and PS_SHAPE_THREADS"
#endif

#define PS_SHAPE_NAME3(b, e, t) shape_u##b##_e##e##_t##t
#define PS_SHAPE_NAME2(b, e, t) PS_SHAPE_NAME3(b, e, t)
#define PS_SHAPE_NAME PS_SHAPE_NAME2(PS_SHAPE_BITS, PS_SHAPE_ITEMS, PS_SHAPE_THREADS)

namespace ps {

template <typename K, int E, int NT> struct ShapeCfg {
    static constexpr int TNT = NT, TE = E, MNT = NT, ME = E, PNT = sizeof(K) == 8 ? 512 : 1024, PE = 8;
    static constexpr int TW = sizeof(K) == 4 ? PS_TILE_WLEV32 : PS_TILE_WLEV64;
};

namespace {
using KeyT = std::conditional_t<PS_SHAPE_BITS == 32, uint32_t, uint64_t>;
using Pipe = Pipeline<KeyT, ShapeCfg<KeyT, PS_SHAPE_ITEMS, PS_SHAPE_THREADS>>;
int run_shape(const SortArgs& a) { return Pipe::run(a); }
size_t ws_shape(const SortArgs& a) { return Pipe::ws_bytes_for(a); }
int run_shape_on(const SortArgs& a, char* ws, size_t cap) { return Pipe::run_on(a, ws, cap); }
}  // namespace

extern const ShapeEntry PS_SHAPE_NAME = {PS_SHAPE_BITS, PS_SHAPE_ITEMS, PS_SHAPE_THREADS, &run_shape, &ws_shape,
                                         &run_shape_on};

}  // namespace ps
