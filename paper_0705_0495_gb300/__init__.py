"""GB300-native PIC-MCC time step for capacitively coupled RF discharges in O2
(Bronold et al., "Radio-frequency discharges in Oxygen. Part 1: Modeling")."""
