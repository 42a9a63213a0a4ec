// FP32-bulk form: state, FFT, exponential and Thomas arithmetic in float;
// tables built in FP64 and rounded once; reductions, the norm and the
// renormalisation scale in FP64.
#include "dgpe_engine.cuh"
namespace dgpe {
Engine *make_engine_f32() { return new EngineT<float>(); }
}
