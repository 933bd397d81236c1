"""GB300-native damped-gradient Skyrme-DFT hot path (arXiv 1610.07522).

The compute path is the C-ABI library ``libsky`` (hand-written CUDA for
sm_103a, declared in ``include/sky.h``); ``binding`` marshals arguments to it
and ``solver`` drives the iteration of Fig. 1 through it.  Importing the
package loads nothing; ``binding.lib()`` loads the library and raises if it
is missing.
"""
