// order_key.cuh -- float <-> unsigned keys whose integer order is the float order, for
// maxima taken with atomicMax.
#pragma once

namespace sfseg {

// Order-preserving map from float to unsigned (larger float -> larger key, negatives below
// positives), so that the maximum is an integer atomicMax.
__device__ __forceinline__ unsigned order_key(float v) {
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float order_value(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

}  // namespace sfseg
