// Instantiation of the float32 SpMM launchers over the (min,+), (max,+) and
// (max,x) semirings.  The (+,x) semiring is the ordinary product of
// inst_f32_f32_f32.cu.
#include "launch.cuh"

namespace spmm {

const Launchers* find_semiring_launchers(int semiring) {
    static const Launchers min_plus = make_launchers<float, float, float, MinPlus>();
    static const Launchers max_plus = make_launchers<float, float, float, MaxPlus>();
    static const Launchers max_times = make_launchers<float, float, float, MaxTimes>();
    switch (semiring) {
        case SPMM_SEMIRING_MIN_PLUS: return &min_plus;
        case SPMM_SEMIRING_MAX_PLUS: return &max_plus;
        case SPMM_SEMIRING_MAX_TIMES: return &max_times;
        default: return nullptr;
    }
}

}  // namespace spmm
