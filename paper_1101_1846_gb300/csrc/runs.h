// How one tick's piece of a serving client runs through several of its
// requests (host-only, tested on the CPU by itself).
//
// A client's requests take consecutive ranges of its sample sequence, so one
// piece of the sequence (one set of batch items, one pass over the client's
// streams) can serve several of them: the bodies write the piece as one
// virtual window of consecutive elements, and the piece's output map
// (gen_body.cuh's OutMap) sends each request's part of the window to that
// request's output, in that request's format.  For the vector stores to stay
// whole, every output must have the same address modulo 32 bytes as its
// place in the window: placement_pad() gives each request an offset whose
// word index is congruent to its first sample's index modulo 8
// (kPhaseWords), so that any window of the client's sequence and all of its
// requests' outputs agree modulo 32 bytes.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace gbrng {

constexpr uint64_t kPhaseWords = 8;

// Bytes to skip from an arena block at byte offset `block` (a multiple of
// 4) so that the output of a request whose first sample is sample `start`
// of its client's sequence begins at a word index congruent to start modulo
// kPhaseWords.  A block of the request's bytes + 4 * (kPhaseWords - 1) always
// has room.
inline uint64_t placement_pad(uint64_t block, uint64_t start)
{
    const uint64_t w = block / 4;
    return 4 * ((start + kPhaseWords - w % kPhaseWords) % kPhaseWords);
}

// A request as the piece builder sees it: its output's byte offset in the
// arena, its size and the samples already written (both in samples), and
// its format.
struct RunReq {
    uint64_t off;
    uint64_t n;
    uint64_t done;
    int fmt;
};

// One segment of a piece: from window index b on, the outputs have format
// fmt and go `shift` elements from their virtual place (origin + index).
struct Seg {
    uint32_t b;
    int fmt;
    int64_t shift;
};

// One client's piece of a tick: a window of m samples whose index 0 is the
// element `origin` (from the arena's base), in segments (the first at b = 0
// with shift 0).  The piece reaches the first `touched` requests; all but
// possibly the last end in it.
struct RunPiece {
    uint64_t origin = 0;
    uint64_t m = 0;
    size_t touched = 0;
    std::vector<Seg> segs;
};

// The piece of at most cap samples (cap < 2^31) that starts with the front
// request's remaining samples and runs on through the following requests
// (whose outputs may be anywhere in the arena).  reqs[0] is the front
// request, reqs[i > 0] have done = 0; count >= 1.  A new segment starts where
// the format or the shift changes (adjacent requests of one format share
// one).  Every shift is a multiple of kPhaseWords (the kernel stores whole
// 16-byte chunks at the shifted places): a request whose output breaks the
// placement rule ends the piece before it.
inline RunPiece run_piece(const RunReq *reqs, size_t count, uint64_t cap)
{
    RunPiece p;
    p.origin = reqs[0].off / 4 + reqs[0].done;
    p.m = std::min(reqs[0].n - reqs[0].done, cap);
    p.touched = 1;
    p.segs.push_back(Seg{0, reqs[0].fmt, 0});
    for (size_t i = 1; i < count && p.m < cap; ++i) {
        const int64_t shift = (int64_t)(reqs[i].off / 4) - (int64_t)(p.origin + p.m);
        if (shift % (int64_t)kPhaseWords != 0)
            break;  // not placed at its sample's phase: it starts a piece of its own
        if (reqs[i].fmt != p.segs.back().fmt || shift != p.segs.back().shift)
            p.segs.push_back(Seg{(uint32_t)p.m, reqs[i].fmt, shift});
        p.m += std::min(reqs[i].n, cap - p.m);
        ++p.touched;
    }
    return p;
}

}  // namespace gbrng
