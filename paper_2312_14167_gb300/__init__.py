"""GB300-native (sm_103a) Flux Reconstruction hot path of the aeroacoustic
shape-optimisation loop of arXiv:2312.14167: the FR residual and explicit RK
step for compressible Navier-Stokes on quad/hex meshes, the observer probe
and the OASPL reduction, batched over the candidate designs of one MADS poll.

The compute path is the C-ABI library ``libfr.so`` (``include/fr.h``); this
package only builds it (``build``) and binds it (``fr``)."""
