"""GB300 (sm_103a) Kalman-filter track fit and combinatorial build step
(arXiv:1705.02876), behind the C interface of include/kf.h."""
