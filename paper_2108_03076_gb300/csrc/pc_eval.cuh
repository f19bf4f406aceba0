// pc_eval.cuh -- the warp-uniform payoff interpreter (eval_path), shared by
// the pricing, portfolio and control-variate kernels.
#pragma once

#include "pc_device.cuh"

namespace pc {
namespace {

// The payoff expression of two paths per lane, all lanes of the warp in step:
// a loop over the executable program, one case per operation (pc_ops.inc).
// (Fetching the next instruction ahead of the current one measured slower:
// it costs a load per instruction the compiler cannot sink.)  `frontier`
// (optional) receives the last generated date ordinal: the window holds the
// simulated dates up to it.
// `hook_` (optional, type PcHook) is called after each generated date.
template <int D, bool GW = false, class PcHook = NoDateHook>
__device__ float2 eval_path(const uint4 *P, const float *pool, float2 *R, const PriceArgs &a,
                            const Rng2 &g, bool live0, bool live1, const float (&Bm)[D * D],
                            const float (&S0)[D], int *frontier = nullptr, PcHook *hook_ = nullptr) {
#include "pc_eval_state.inc"
#define NEXT      \
  {               \
    ++pc;         \
    I = P[pc];    \
    break;        \
  }
#define JUMP_TO(t) \
  {                \
    pc = (t);      \
    I = P[pc];     \
    break;         \
  }
#define JUMP_Z JUMP_TO(int(I.z))
#define JUMP_W JUMP_TO(int(I.w))
#define JUMP_2 JUMP_TO(pc + 2)
#define NEXT_INSN P[pc + 1]
#define ENSURE(o) ensure(o)
  uint4 I = P[0];
  for (;;) {
    switch (I.x & 0xffu) {
#include "pc_ops.inc"
    }
  }
#undef NEXT
#undef JUMP_TO
#undef JUMP_Z
#undef JUMP_W
#undef JUMP_2
#undef NEXT_INSN
#undef ENSURE
#undef PUSH
#undef STK
#undef BINF
#undef BINI
#undef IMM
#undef GEN_DATE
#undef FUSED_VALUE
#undef FUSED_TEST
}

}  // namespace
}  // namespace pc
