// K7: hand-written adjoint of ln L (in progress).
#include "runtime.cuh"

namespace chim {

int backward(Ctx &, Catalog &, Workspace &, int, int) {
    set_error("gradient not available in this build");
    return CHIMERA_ERR_UNSUPPORTED;
}

}  // namespace chim
