// lbm_fp64.cu -- FP64 mode: FP64 arithmetic and storage, every formula in the
// fixed operation order of the FP64 CPU oracle (built with --fmad=false).
#include "lbm_launch.cuh"

namespace lbm {

cudaError_t launch_init_p0(int Q, const Params &p, void *dst, void *mac, const uint8_t *flags, const double u0[3],
                           cudaStream_t s) {
    return Q == 9 ? init_t<Lat<9>, PF64>(p, dst, mac, flags, u0, s) : init_t<Lat<19>, PF64>(p, dst, mac, flags, u0, s);
}
cudaError_t launch_load_p0(int Q, const Params &p, const double *stage, long long c0, long long n, void *dst,
                           void *mac, const uint8_t *flags, cudaStream_t s) {
    return Q == 9 ? load_t<Lat<9>, PF64>(p, stage, c0, n, dst, mac, flags, s)
                  : load_t<Lat<19>, PF64>(p, stage, c0, n, dst, mac, flags, s);
}
cudaError_t launch_macros_p0(int Q, const Params &p, const void *src, const uint16_t *owner, long long c0,
                             long long n, double *out, cudaStream_t s) {
    return Q == 9 ? macros_t<Lat<9>, PF64>(p, src, owner, c0, n, out, s)
                  : macros_t<Lat<19>, PF64>(p, src, owner, c0, n, out, s);
}
cudaError_t launch_links_p0(int Q, const Params &p, const StepBufs &sb, int grid, cudaStream_t s) {
    return Q == 9 ? links_t<Lat<9>, PF64>(p, sb, grid, s) : links_t<Lat<19>, PF64>(p, sb, grid, s);
}
cudaError_t launch_bulk_p0(int Q, const Params &p, const StepBufs &sb, cudaStream_t s) {
    return Q == 9 ? bulk_t<Lat<9>, PF64>(p, sb, s) : bulk_t<Lat<19>, PF64>(p, sb, s);
}
cudaError_t launch_finish_p0(int Q, const Params &p, const StepBufs &sb, cudaStream_t s) {
    return Q == 9 ? finish_t<Lat<9>, PF64>(p, sb, s) : finish_t<Lat<19>, PF64>(p, sb, s);
}

} // namespace lbm
