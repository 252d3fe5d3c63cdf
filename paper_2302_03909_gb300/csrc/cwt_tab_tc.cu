// Pass-2 tile-pipeline instantiations: tensor-core forms (cwt_tc.cuh) and FP32 (cwt_f32tile.cuh).
#include "cwt_tables.cuh"
#include "cwt_tc.cuh"
#include "cwt_f32tile.cuh"

namespace cwtk {

template <int FORM, bool CROP>
static TcEntry tc_entry() {
    return {k_wide2_tma<FORM, CROP>, k_wide2_tc_g<FORM, CROP>, tma_threads(FORM), tma_smem_bytes(FORM),
            tc_smem_bytes(FORM)};
}

void fill_tc_tables(Tables& t) {
    t.wide2_tc[TC_FP16][0] = tc_entry<TC_FP16, false>();
    t.wide2_tc[TC_FP16][1] = tc_entry<TC_FP16, true>();
    t.wide2_tc[TC_BF16][0] = tc_entry<TC_BF16, false>();
    t.wide2_tc[TC_BF16][1] = tc_entry<TC_BF16, true>();
    t.wide2_tc[TC_FP16X3][0] = tc_entry<TC_FP16X3, false>();
    t.wide2_tc[TC_FP16X3][1] = tc_entry<TC_FP16X3, true>();
    t.wide2_tc[TC_BF16X3][0] = tc_entry<TC_BF16X3, false>();
    t.wide2_tc[TC_BF16X3][1] = tc_entry<TC_BF16X3, true>();
    // FP32 arithmetic on the same tile pipeline (precision 0)
    t.wide2_tc[0][0] = {k_wide2_f32<false>, k_wide2_f32_g<false>, kF32Threads, f32_smem_bytes(true),
                        f32_smem_bytes(false)};
    t.wide2_tc[0][1] = {k_wide2_f32<true>, k_wide2_f32_g<true>, kF32Threads, f32_smem_bytes(true),
                        f32_smem_bytes(false)};
}

}  // namespace cwtk
