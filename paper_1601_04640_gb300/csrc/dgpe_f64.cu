// FP64 form: every substep in double precision.
#include "dgpe_engine.cuh"
namespace dgpe {
Engine *make_engine_f64() { return new EngineT<double>(); }
}
