// lbm_fp32.cu -- reduced-precision modes: FP32 arithmetic with populations
// stored as deviations f - w in FP32 (p1) or FP16 (p2).
#include "lbm_launch.cuh"
#include "lbm_bnd.cuh"

namespace lbm {

cudaError_t launch_init_p12(int Q, int prec, const Params &p, void *dst, void *mac, const uint8_t *flags,
                            const double u0[3], cudaStream_t s) {
    if (prec == 1)
        return Q == 9 ? init_t<Lat<9>, PF32>(p, dst, mac, flags, u0, s) : init_t<Lat<19>, PF32>(p, dst, mac, flags, u0, s);
    return Q == 9 ? init_t<Lat<9>, PF16>(p, dst, mac, flags, u0, s) : init_t<Lat<19>, PF16>(p, dst, mac, flags, u0, s);
}
cudaError_t launch_load_p12(int Q, int prec, const Params &p, const double *stage, long long c0, long long n,
                            void *dst, void *mac, const uint8_t *flags, cudaStream_t s) {
    if (prec == 1)
        return Q == 9 ? load_t<Lat<9>, PF32>(p, stage, c0, n, dst, mac, flags, s)
                      : load_t<Lat<19>, PF32>(p, stage, c0, n, dst, mac, flags, s);
    return Q == 9 ? load_t<Lat<9>, PF16>(p, stage, c0, n, dst, mac, flags, s)
                  : load_t<Lat<19>, PF16>(p, stage, c0, n, dst, mac, flags, s);
}
cudaError_t launch_macros_p12(int Q, int prec, const Params &p, const void *src, const uint16_t *owner, long long c0,
                              long long n, double *out, cudaStream_t s) {
    if (prec == 1)
        return Q == 9 ? macros_t<Lat<9>, PF32>(p, src, owner, c0, n, out, s)
                      : macros_t<Lat<19>, PF32>(p, src, owner, c0, n, out, s);
    return Q == 9 ? macros_t<Lat<9>, PF16>(p, src, owner, c0, n, out, s)
                  : macros_t<Lat<19>, PF16>(p, src, owner, c0, n, out, s);
}
cudaError_t launch_links_p12(int Q, int prec, const Params &p, const StepBufs &sb, int grid, cudaStream_t s) {
    if (prec == 1) return Q == 9 ? links_t<Lat<9>, PF32>(p, sb, grid, s) : links_t<Lat<19>, PF32>(p, sb, grid, s);
    return Q == 9 ? links_t<Lat<9>, PF16>(p, sb, grid, s) : links_t<Lat<19>, PF16>(p, sb, grid, s);
}
cudaError_t launch_bulk_p12(int Q, int prec, const Params &p, const StepBufs &sb, cudaStream_t s) {
    if (prec == 1) return Q == 9 ? bulk_t<Lat<9>, PF32>(p, sb, s) : bulk_t<Lat<19>, PF32>(p, sb, s);
    return Q == 9 ? bulk_t<Lat<9>, PF16>(p, sb, s) : bulk_t<Lat<19>, PF16>(p, sb, s);
}
cudaError_t launch_finish_p12(int Q, int prec, const Params &p, const StepBufs &sb, cudaStream_t s) {
    if (prec == 1) return Q == 9 ? finish_t<Lat<9>, PF32>(p, sb, s) : finish_t<Lat<19>, PF32>(p, sb, s);
    return Q == 9 ? finish_t<Lat<9>, PF16>(p, sb, s) : finish_t<Lat<19>, PF16>(p, sb, s);
}

cudaError_t launch_bnd(int Q, int prec, const Params &p, const BndArgs &a, const StepBufs &sb, int grid,
                       cudaStream_t s) {
    if (prec == 1) return Q == 9 ? bnd_t<Lat<9>, PF32>(p, a, sb, grid, s) : bnd_t<Lat<19>, PF32>(p, a, sb, grid, s);
    return Q == 9 ? bnd_t<Lat<9>, PF16>(p, a, sb, grid, s) : bnd_t<Lat<19>, PF16>(p, a, sb, grid, s);
}

} // namespace lbm
