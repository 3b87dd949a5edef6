// Lane layout of the FP32 passes: a lane loads 16 B (four floats) of a
// node's tile row; L lanes cover the row, a warp gathers 32 / L edges a step.
#pragma once

namespace ppr {

template <int KT>
struct Lay32 {
  static constexpr int V = KT >= 4 ? 4 : KT;  // floats per lane load (16 B when 4)
  static constexpr int L = KT / V;            // lanes covering one row of the tile
  static constexpr int EPW = 32 / L;
};

template <int V>
__device__ __forceinline__ void ldf(const float* p, float (&v)[V]) {
  if constexpr (V == 4) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (V == 2) {
    float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
  } else {
    v[0] = __ldg(p);
  }
}

}  // namespace ppr
