// output.cu -- the pair buffer of a materialising join and its final compaction.
//
// Warps fill whole chunks of kChunkPairs slots (emit.cuh); each warp's last chunk
// is usually partly used.  After the join kernels finish, the host reads the
// recorded partial chunks, pairs the holes below `count` with the valid pairs at
// or above `count`, and one small kernel moves those pairs, so that
// pairs[0, count) is dense.  The moved volume is at most one chunk per warp.
#include <algorithm>
#include <memory>
#include <vector>

#include "emit.cuh"
#include "engine.cuh"

namespace hj {

struct Move {
    unsigned long long src, dst, len;
};

template <class P>
__global__ void move_pairs_kernel(P *pairs, const Move *moves, uint64_t nmoves) {
    for (uint64_t m = blockIdx.x; m < nmoves; m += gridDim.x) {
        const Move mv = moves[m];
        for (uint64_t i = threadIdx.x; i < mv.len; i += blockDim.x) pairs[mv.dst + i] = pairs[mv.src + i];
    }
}

hj_status PairSink::reset(uint64_t cap_pairs) {
    areas.clear();
    caps.clear();
    pcap = cap_pairs ? cap_pairs : 1;
    return pairs.alloc(pcap * 2ull * width);
}

hj_status PairSink::new_area(uint64_t warps, RecArea *ra) {
    auto b = std::make_unique<DevBuf>(c);
    HJ_TRY(b->alloc(16 + warps * sizeof(ChunkRec)));
    HJ_CUDA(c, cudaMemsetAsync(b->p, 0, 16, c->stream));
    ra->n = (unsigned long long *)b->p;
    ra->rec = (ChunkRec *)((char *)b->p + 16);
    ra->cap = warps;
    areas.push_back(std::move(b));
    caps.push_back(warps);
    return HJ_OK;
}

hj_status PairSink::finalize(uint64_t count, uint64_t cursor) {
    if (cursor > pcap) return set_err(c, HJ_E_CUDA, "pair cursor %llu beyond capacity %llu",
                                      (unsigned long long)cursor, (unsigned long long)pcap);
    if (count == cursor) return HJ_OK;
    std::vector<ChunkRec> recs;
    for (size_t i = 0; i < areas.size(); ++i) {
        unsigned long long n = 0;
        HJ_CUDA(c, cudaMemcpyAsync(&n, areas[i]->p, 8, cudaMemcpyDeviceToHost, c->stream));
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
        n = std::min<unsigned long long>(n, caps[i]);
        size_t old = recs.size();
        recs.resize(old + n);
        if (n)
            HJ_CUDA(c, cudaMemcpyAsync(recs.data() + old, (char *)areas[i]->p + 16, n * sizeof(ChunkRec),
                                       cudaMemcpyDeviceToHost, c->stream));
    }
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    // holes [base + used, base + kChunkPairs), sorted
    std::vector<std::pair<uint64_t, uint64_t>> holes;
    for (auto &r : recs)
        if (r.used < kChunkPairs) holes.push_back({r.base + r.used, r.base + kChunkPairs});
    std::sort(holes.begin(), holes.end());
    // holes below count, and valid ranges in [count, cursor)
    std::vector<std::pair<uint64_t, uint64_t>> dst, src;
    uint64_t at = count;
    for (auto &h : holes) {
        if (h.first < count) dst.push_back({h.first, std::min<uint64_t>(h.second, count)});
        uint64_t a = std::max<uint64_t>(h.first, count);
        if (a > at) src.push_back({at, a});
        if (h.second > at) at = std::max<uint64_t>(at, h.second);
    }
    if (cursor > at) src.push_back({at, cursor});
    uint64_t nd = 0, ns = 0;
    for (auto &d : dst) nd += d.second - d.first;
    for (auto &s : src) ns += s.second - s.first;
    if (nd != ns)
        return set_err(c, HJ_E_CUDA, "output compaction mismatch: %llu holes, %llu tail pairs",
                       (unsigned long long)nd, (unsigned long long)ns);
    std::vector<Move> moves;
    size_t i = 0, j = 0;
    uint64_t di = dst.empty() ? 0 : dst[0].first, sj = src.empty() ? 0 : src[0].first;
    while (i < dst.size() && j < src.size()) {
        uint64_t len = std::min(dst[i].second - di, src[j].second - sj);
        moves.push_back({sj, di, len});
        di += len;
        sj += len;
        if (di == dst[i].second && ++i < dst.size()) di = dst[i].first;
        if (sj == src[j].second && ++j < src.size()) sj = src[j].first;
    }
    if (moves.empty()) return HJ_OK;
    DevBuf dm(c);
    HJ_TRY(dm.alloc(moves.size() * sizeof(Move)));
    HJ_CUDA(c, cudaMemcpyAsync(dm.p, moves.data(), moves.size() * sizeof(Move), cudaMemcpyHostToDevice, c->stream));
    unsigned grid = (unsigned)std::min<size_t>(moves.size(), (size_t)num_sms(c) * 8);
    if (width == 4)
        HJ_LAUNCH(c, "pairs_compact", move_pairs_kernel<uint2>, grid, 256, 0, (uint2 *)pairs.p, dm.as<Move>(),
                  (uint64_t)moves.size());
    else
        HJ_LAUNCH(c, "pairs_compact", move_pairs_kernel<ulonglong2>, grid, 256, 0, (ulonglong2 *)pairs.p,
                  dm.as<Move>(), (uint64_t)moves.size());
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));  // `moves` is a host temporary
    return HJ_OK;
}

}  // namespace hj
