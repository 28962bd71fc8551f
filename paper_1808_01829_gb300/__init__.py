"""GB300 block multishift RHMC: SBCGrQ solves and the pseudofermion force.

Hot path of de Forcrand & Keegan, arXiv:1808.01829, as hand-written CUDA for
sm_103a behind the C ABI in include/rhmc.h (librhmc.so).  Submodules:

* ``api``        torch-facing binding of the C ABI (RhmcContext)
* ``functional`` the same entry points as functions of the link tensor
                 (apply_mdagm, block_multishift_cg, force, PseudofermionAction.apply)
* ``action``     torch.autograd.Function for the pseudofermion action / force
* ``remez``      rational approximation coefficients of Eq. (RA) (host set-up)
* ``synthetic``  seeded synthetic gauge fields and pseudofermions
* ``_build``     in-tree nvcc build of librhmc.so

Importing the package does not load the CUDA library; the first use of
``RhmcContext`` does, and fails loudly if it is missing.
"""

__all__ = ["RhmcContext", "PseudofermionAction"]


def __getattr__(name):
    if name == "RhmcContext":
        from .api import RhmcContext

        return RhmcContext
    if name == "PseudofermionAction":
        from .action import PseudofermionAction

        return PseudofermionAction
    raise AttributeError(name)
