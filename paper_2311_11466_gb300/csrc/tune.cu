// Autotuner of launch shapes (no counterpart in the paper; it changes no
// arithmetic).  The first iteration of a context whose kind of scan -- device,
// pattern side N and J bucket (floor(log2 J)) -- has not been seen in this
// process times the candidate launch shapes of the concur step on the
// context's own data, keeps the fastest and caches the choice for every later
// context of that kind:
//   object gather: tile shapes 16 x 32, 8 x 32, 32 x 32 and 8 x 64 pixels;
//   probe partial pass: 1 or 2 probe pixels per thread (16-byte loads of y).
// Every candidate adds the same terms in the same order per pixel, so the
// results are bit-identical whichever shape wins; only the time differs.
//
// The 128^2 cluster shape of the divide step is chosen the same way, at the
// load of a scan (tune_divide128): the candidates are clusters of 8 CTAs of
// 128 threads and of 16 CTAs of 64 threads (the same 16 x 8 radix split, so
// the same arithmetic), each timed on the scan's own data in the error-only
// mode, which writes nothing the iteration reads.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace ptycho {
namespace {

std::mutex g_mu;
std::map<std::tuple<int, int, int>, TuneChoice> g_cache;

int j_bucket(int J) {
    int b = 0;
    while (b < 30 && (1 << (b + 1)) <= J) ++b;
    return b;
}

constexpr int kReps = 3;

// Average ms of kReps launches of fn() on st (after one untimed launch).
template <class F>
cudaError_t time_ms(cudaStream_t st, F fn, float* ms) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    if ((e = fn()) == cudaSuccess && (e = cudaEventRecord(e0, st)) == cudaSuccess) {
        for (int i = 0; i < kReps && e == cudaSuccess; ++i) e = fn();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        *ms /= kReps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

cudaError_t upload_csr(const int32_t* pos_rc, int J, int N, int Mr, int Mc, int shape, ConcurBufs& cb,
                       cudaStream_t st) {
    std::vector<int> ptr;
    std::vector<int4> list;
    const TileShape sh = kGatherShape[shape];
    build_tile_csr(pos_rc, J, N, Mr, Mc, sh, ptr, list);
    cudaError_t e = cudaMemcpyAsync(cb.tile_ptr, ptr.data(), ptr.size() * sizeof(int),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !list.empty())
        e = cudaMemcpyAsync(cb.tile_win, list.data(), list.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
    cb.tiles_r = (Mr + sh.rows - 1) / sh.rows;
    cb.tiles_c = (Mc + sh.cols - 1) / sh.cols;
    cb.gather_shape = shape;
    return e;
}

}  // namespace

TuneChoice tune_lookup(int device, int N, int J) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find({device, N, j_bucket(J)});
    if (it != g_cache.end()) return it->second;
    return TuneChoice{};
}

cudaError_t tune_concur(int device, ConcurScan& cs, const int32_t* pos_rc_host, cudaStream_t st,
                        TuneChoice* out) {
    ConcurBufs& cb = cs.cb;
    const int J = cs.J, N = cs.N, Mr = cs.Mr, Mc = cs.Mc;
    TuneChoice c = tune_lookup(device, N, J);
    cudaError_t e = cudaSuccess;
    if (!c.valid) {
        // the divide step of this iteration has written y: wait for it untimed
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        for (int s = 0; s < kGatherShapes; ++s) {
            if ((e = upload_csr(pos_rc_host, J, N, Mr, Mc, s, cb, st)) != cudaSuccess) return e;
            e = time_ms(st, [&] { return launch_gather(cs, st); }, &c.gather_ms[s]);
            if (e != cudaSuccess) return e;
        }
        int best = 0;
        for (int s = 1; s < kGatherShapes; ++s)
            if (c.gather_ms[s] < c.gather_ms[best]) best = s;
        c.gather_shape = best;
        for (int p = 1; p <= 2; ++p) {
            ConcurScan t = cs;
            t.cb.probe_ppt = p;
            e = time_ms(st, [&] { return launch_probe_partial(t, st); }, &c.probe_ms[p - 1]);
            if (e != cudaSuccess) return e;
        }
        c.probe_ppt = c.probe_ms[1] < c.probe_ms[0] ? 2 : 1;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            const auto key = std::make_tuple(device, N, j_bucket(J));
            auto it = g_cache.find(key);
            if (it != g_cache.end()) {
                c.divide_tuned = it->second.divide_tuned;      // chosen at load
                c.divide_variant = it->second.divide_variant;
                c.divide_ms[0] = it->second.divide_ms[0];
                c.divide_ms[1] = it->second.divide_ms[1];
            }
            c.valid = true;
            g_cache[key] = c;
        }
    }
    // this context: the chosen shapes (the device holds the tile lists of
    // cb.gather_shape: the one built at load, or the last candidate timed)
    if (cb.gather_shape != c.gather_shape)
        if ((e = upload_csr(pos_rc_host, J, N, Mr, Mc, c.gather_shape, cb, st)) != cudaSuccess) return e;
    cb.probe_ppt = c.probe_ppt;
    if (out) *out = c;
    return cudaSuccess;
}

cudaError_t tune_apply_shape(const int32_t* pos_rc_host, int J, int N, int Mr, int Mc, int shape,
                             ConcurBufs& cb, cudaStream_t st) {
    return upload_csr(pos_rc_host, J, N, Mr, Mc, shape, cb, st);
}

void tune_store_divide(int device, int N, int J, int variant, const float ms[2]) {
    std::lock_guard<std::mutex> lk(g_mu);
    TuneChoice& c = g_cache[{device, N, j_bucket(J)}];
    c.divide_variant = variant;
    c.divide_ms[0] = ms[0];
    c.divide_ms[1] = ms[1];
    c.divide_tuned = true;
}

}  // namespace ptycho
