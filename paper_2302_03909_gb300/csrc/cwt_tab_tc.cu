// Tensor-core pass-2 instantiations (see cwt_tc.cuh and cwt_tables.cuh).
#include "cwt_tables.cuh"
#include "cwt_tc.cuh"

namespace cwtk {

template <int FORM, bool CROP>
static TcEntry tc_entry() { return {k_wide2_tma<FORM, CROP>, k_wide2_tc_g<FORM, CROP>, tma_threads(FORM)}; }

void fill_tc_tables(Tables& t) {
    t.wide2_tc[TC_FP16][0] = tc_entry<TC_FP16, false>();
    t.wide2_tc[TC_FP16][1] = tc_entry<TC_FP16, true>();
    t.wide2_tc[TC_BF16][0] = tc_entry<TC_BF16, false>();
    t.wide2_tc[TC_BF16][1] = tc_entry<TC_BF16, true>();
    t.wide2_tc[TC_FP16X3][0] = tc_entry<TC_FP16X3, false>();
    t.wide2_tc[TC_FP16X3][1] = tc_entry<TC_FP16X3, true>();
    t.wide2_tc[TC_BF16X3][0] = tc_entry<TC_BF16X3, false>();
    t.wide2_tc[TC_BF16X3][1] = tc_entry<TC_BF16X3, true>();
}

}  // namespace cwtk
