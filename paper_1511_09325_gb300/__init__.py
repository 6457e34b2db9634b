"""GB300-native spiking cortical-column simulator (arxiv 1511.09325)."""
